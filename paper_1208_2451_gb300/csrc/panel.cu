// Panel factorization of LU_PRRP: strong rank revealing QR of the transposed m x w panel
// (Algorithm 2 of Appendix A, applied as in Algorithm 1, lines 3-4).
//
// One persistent grid owns the panel: CTA c holds a contiguous chunk of panel rows in
// shared memory for the whole kernel, so the panel is read from HBM once.  In the paper's
// notation B = panel^T, so a panel row is a column of B.
//
// QR with column pivoting, step t:
//   * every CTA proposes its row of largest remaining squared norm ||B(t:w, q)||^2 (ties to
//     the smallest position), with that row's values and its exact squared norm;
//   * the proposals are exchanged (below) and every CTA takes the same winner p and builds
//     the same Householder reflector from its values, H = I - beta v v^T with
//     H x = alpha e_1, alpha = -sign(x_1) ||x||;
//   * the winner takes position t (the row at position t moves to the winner's position),
//     R(0:t, t) and R(t, t) = alpha are recorded, and H is applied to every remaining row
//     with a team of lanes per row (shuffle reductions).  Remaining norms are downdated,
//     ||B(t+1:w, q)||^2 = ||B(t:w, q)||^2 - B(t, q)^2, and recomputed from the values
//     whenever they fall below 1e-4 of their last exact value, which keeps their relative
//     error near 1e-12.
// Then M = R11^-1 R12 for each remaining row by back substitution.  While the largest
// |M_ij| exceeds tau (ties to the smallest j, then i), selected slot i and remaining row j
// are interchanged; instead of a new QR, M is updated by the exact basis-exchange formulas
// (mu = M_ij, c = M(:, j)):  M'(k, r) = M(k, r) - M(i, r) c_k / mu,  M'(i, r) = M(i, r) / mu,
// and the row leaving the selection gets M'(:, j) = -c / mu with M'(i, j) = 1 / mu.
// Each interchange raises |det R11| by |mu| > tau, so the loop ends (Appendix A).
//
// Latency structure of a QRCP step.  On this GPU an FP64 instruction holds its
// sub-partition's FP64 unit for 64 cycles whatever its active lanes, and a square root
// with a division costs about 1200 cycles, so the step is arranged around three warps'
// roles.  Warp 0 of each CTA only communicates, warp 1 (the helper) only forms the
// reflector of the CTA's own candidate, and the other warps own the rows.  A row warp
// applies the step's reflector in two parts: first the dot product, the new B(t, q), the
// norm downdate and the proposal for the next step (the critical part), then, while warp
// 0 exchanges the proposals, the rest of the row update B(t+1:w, q) -= f v(t+1:w) (each
// warp finishes its own proposed row first, since that row's values are published).  The
// arithmetic is the same as applying the whole reflector before proposing.  Rows are
// spread so that every FP64 unit of the SM gets the same share.
//
// Exchange, grid form (one cooperative grid): key arrays (a step's keys contiguous) and
// record arrays rotate over kQSlots steps, all keys absent (0) and all record words
// sentinels (a NaN that finite data never produces) at launch.  At step t a CTA writes its
// proposed row into its record with plain stores and its 64-bit key (below) with a
// relaxed store; the helper warp computes the candidate's alpha and beta and writes them
// into the record.  Warp 0 of every CTA polls all keys until every key of the step is
// present, takes the largest, and reads again any word of the winner's record that still
// holds the sentinel.  Right after publishing, it prepares its slot of step t - 2 (every
// reader of it has published step t - 1 since) for the slot's next use: key absent,
// record sentinels.  One
// fence every kQFenceEvery steps orders those preparations before the slot's reuse for
// every reader, so no stale key or record word is ever taken, and no store waits on the
// critical path for another store to complete.
// Exchange, cluster form (m <= 512 by default): the grid is one thread-block cluster;
// each CTA pushes its key into every CTA's shared memory and arrives on that CTA's
// mbarrier; the winner's row, alpha and beta are read directly from the winning CTA's
// shared memory, with the same sentinel rule.
//
// The reflector of the winning row is computed by the winner's helper warp alone, so all
// CTAs apply the same bits.
//
// Outputs: L21 = M^T (row w + r of the final order -> L21 row r), the final position of
// every panel row, and a list of (destination, source) row moves for the permute kernel.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "select.cuh"

namespace prrp {

using namespace sel;

namespace {

constexpr int kThreads = kPanelThreads;            // communication, helper and row warps
constexpr int kWarps = kThreads / 32;
constexpr int kRowWarps = kWarps - 2;
constexpr int kRowWarp0 = 2;                       // first row warp
constexpr int kBarProp = 1;                        // named barriers: proposals gathered,
constexpr int kBarWin = 2;                         //   winner of the step published,
constexpr int kBarHelp = 3;                        //   this CTA's record published
constexpr int kPollSlots = (kPanelMaxCtas + 31) / 32;
// A record word not written yet: all bits set, a NaN that finite data never produces (the
// host fills every record slot with 0xFF bytes at launch, the kernel refills a slot for
// its reuse).
constexpr unsigned long long kSentinel = ~0ull;

// Cooperative panel grids from different streams or contexts must not be resident at the
// same time: two partially resident grids could each wait at their grid barrier for CTAs
// that the other one keeps off the SMs.  Every panel launch on a device therefore waits
// for the previous one (on any stream) through this per-device event chain; other kernels
// still overlap with them freely.
std::mutex g_coop_mu;
cudaEvent_t g_coop_done[64] = {};

// Lanes per row team for panels of width class W.  With up to ~190 rows per CTA, teams of
// 4 lanes (8 at W = 128) fill whole warp passes on several sub-partitions, two warps each;
// with more rows, one lane per row (2 at W = 128) needs about 40% fewer FP64 instructions
// per row (no team reductions, no per-row fixed cost) and still keeps two row warps on
// most sub-partitions (measured: 20% faster at 256 rows per CTA, 9% slower at 108).
__host__ __device__ constexpr int panel_team(int W, bool many_rows) {
  return many_rows ? (W >= 128 ? 2 : 1) : (W >= 128 ? 8 : 4);
}
constexpr int kManyRows = 192;     // rows per CTA from which the one-lane-per-row form runs

// ---- global-memory signalling (grid form) ----
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ double ld_relaxed_f64(const double* p) {
  return vval(ld_relaxed_u64(reinterpret_cast<const unsigned long long*>(p)));
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// ---- named barriers between the communication warp and the row warps ----
__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// ---- distributed shared memory of a thread-block cluster (cluster form) ----
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint32_t cl_map(const void* p, unsigned rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_addr(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ double cl_ld_f64(uint32_t a) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ int2 cl_ld_int2(uint32_t a) {
  int2 v;
  asm volatile("ld.shared::cluster.v2.s32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void cl_st_u64(uint32_t a, unsigned long long v) {
  asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}
__device__ __forceinline__ void cl_st_s32(uint32_t a, int v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void cl_arrive(uint32_t a) {
  asm volatile("red.release.cluster.shared::cluster.add.u32 [%0], 1;" ::"r"(a) : "memory");
}
__device__ __forceinline__ unsigned cl_ld_acquire(uint32_t a) {
  unsigned v;
  asm volatile("ld.acquire.cluster.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void cl_fence() { asm volatile("fence.acq_rel.cluster;" ::: "memory"); }
// every thread of every CTA of the cluster (hardware barrier)
__device__ __forceinline__ void cl_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// arrive on another CTA's mbarrier (release at cluster scope covers this thread's stores)
__device__ __forceinline__ void mbar_arrive_remote(uint32_t bar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cluster(unsigned long long* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

}  // namespace

// Layout: warp 0 communicates, warp 1 forms reflectors; row warp k (warp k + 2) owns a
// fixed slice of the CTA's rows for the whole kernel, and inside a warp teams of TEAM = 4
// lanes (8 for W = 128) work on one row each.  Whole warp passes of rows go to the row
// warps in order, which puts consecutive passes on different sub-partitions.  All per-row
// state (values, remaining squared norm, position, pending update) is touched only by its
// own warp during the QRCP loop.  (TEAM = 1 or 2 for CTAs with many rows, see panel_team.)
//
// CL = false: one cooperative grid; QRCP proposals through the rotating key arrays, the
// interchange test through exchange records and a counter barrier in global memory.
// CL = true: the grid is one thread-block cluster; QRCP keys are pushed into every CTA's
// shared memory behind an mbarrier, the interchange test uses a counter in CTA 0 (remote
// atomics), and rows are read from the other CTAs' shared memory.  The cluster's CTAs are
// co-scheduled by the hardware, so cluster-form panels from different streams may run at
// the same time.  In the cluster form no CTA leaves before the others are done reading its
// shared memory (a hardware cluster barrier ends the kernel), and every decision that ends
// a loop is taken identically by all CTAs from the same exchanged data.
template <int W, bool CL, int TEAM>
__global__ void __launch_bounds__(kThreads, 1) panel_rrqr_kernel(PanelParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int TPW = 32 / TEAM;     // rows per warp pass
  constexpr int SP = W + TEAM;       // row stride: a warp pass touches each bank pair evenly
  constexpr int NV = (W + 31) / 32;  // row values per lane of warp 0
  __shared__ Cand s_wc[kWarps];
  __shared__ int s_ok;
  __shared__ int s_abort;
  __shared__ double s_v[2][W];                       // the step's reflector vector v (QRCP) /
                                                      //   the winning row (interchanges)
  __shared__ double s_beta[2];
  __shared__ double s_ab[CL ? 2 : 1][2];            // cluster form: this CTA's alpha, beta
  __shared__ int s_pw[2];
  __shared__ int s_qok[2];
  __shared__ Cand s_gbest;
  // cluster form: QRCP keys pushed by every CTA (two step parities), their mbarriers,
  // and the interchange records (value, tie-breaks, row) read by the others
  __shared__ unsigned long long s_rk[CL ? 2 * 16 : 1];
  __shared__ int s_raux[CL ? 2 * 16 : 1];
  __shared__ __align__(8) unsigned long long s_mb[CL ? 2 : 1];
  __shared__ double s_xval[CL ? 2 : 1];
  __shared__ int2 s_xkey[CL ? 2 : 1];
  __shared__ double s_xrow[CL ? 2 * W : 1];
  __shared__ unsigned s_ctr;

  DevState* st = p.st;
  const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  if constexpr (!CL) {
    if (tid == 0) s_abort = dev_status(st) != 0;     // one decision for the whole CTA
    __syncthreads();
    if (s_abort) return;
  } else {
    if (tid == 0) {
      s_ctr = 0;
      mbar_init(&s_mb[0], G);
      mbar_init(&s_mb[1], G);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    cl_sync_all();                                  // counter and barriers ready, every CTA running
  }
  {

  const int tl = lane & (TEAM - 1), tw = lane / TEAM;            // lane in team, team in warp
  const unsigned tmask = (TEAM == 32 ? 0xffffffffu : ((1u << TEAM) - 1u)) << (lane & ~(TEAM - 1));
  const int w = p.w, m = p.m;
  const int rpc = p.rows_per_cta;
  const int r0 = cta * rpc;
  const int nr = max(0, min(rpc, m - r0));
  // rows per row warp: whole warp passes
  const int rpw = ((nr + kRowWarps - 1) / kRowWarps + TPW - 1) / TPW * TPW;
  const int rw = warp - kRowWarp0;                                // row warp index
  const int wr0 = rw < 0 ? 0 : min(nr, rw * rpw), wr1 = rw < 0 ? 0 : min(nr, wr0 + rpw);
  const unsigned limit = st->spin_limit ? st->spin_limit : kSpinLimit;

  double* Ps = reinterpret_cast<double*>(smem_raw);      // rpc x SP panel rows
  double* Rs = Ps + (size_t)rpc * SP;                     // W x W, R11 (row-major)
  double* nrm = Rs + W * W;                               // rpc remaining squared norms
  double* thr = nrm + rpc;                                // rpc recompute thresholds
  double* fpend = thr + rpc;                              // rpc pending reflector factors
  double* rdiag = fpend + rpc;                            // W reciprocals of diag(R11)
  int* pos = reinterpret_cast<int*>(rdiag + W);           // rpc current positions
  int* pend = pos + rpc;                                  // rpc: rest of the update pending

  __syncthreads();
  if (tid == 0) s_abort = 0;
  for (int e = tid; e < nr * w; e += blockDim.x) {
    const int r = e / w, c = e - r * w;
    Ps[r * SP + c] = p.P[(long long)(r0 + r) * p.ldp + c];
  }
  __syncthreads();

  // ---------------- QR with column pivoting ----------------
  if (warp == 0) {
    // ---- communication warp ----
    for (int t = 0; t < w; ++t) {
      const int par = t & 1;
      named_sync(kBarProp, kThreads);                // the row warps' proposals for step t
      Cand d = (lane >= kRowWarp0 && lane < kWarps) ? s_wc[lane] : Cand{0ull, 0, 0, -1};
      d = warp_max_key(d);
      const bool has = d.v > kNoCand && d.aux >= 0;
      int ok = 1;
      Cand g{0ull, 0, 0, -1};
      double xv[NV];
#pragma unroll
      for (int k = 0; k < NV; ++k) xv[k] = 0.0;
      double alpha = 0.0, beta = 0.0;
      if constexpr (!CL) {
        const int q = t % kQSlots;
        const size_t slot = (size_t)q * G + cta;
        double* rec = p.qrow + slot * kQStride;
        // The key is a relaxed store: this CTA's absent key and sentinel record of slot q,
        // prepared kQSlots - 2 steps ago, are ordered before it by an exchange fence since
        // (the host prepared every slot's first use before the launch).  The record's
        // values need no ordering: a reader takes a word once it no longer holds the
        // sentinel.
        if (has)
          for (int i = lane; i < w; i += 32) rec[i] = Ps[d.aux * SP + i];
        __syncwarp();
        if (lane == 0) st_relaxed_u64(p.qkey + slot * kQKeyStride, has ? d.v : kNoCand);
        named_arrive(kBarHelp, 64);                   // the helper may fill in alpha, beta
        if (t >= 2 && t - 2 + kQSlots < w) {
          // the slot of step t - 2, whose readers have all published step t - 1 since: its
          // key absent and its record sentinels again, for step t - 2 + kQSlots
          const size_t s2 = (size_t)((t - 2) % kQSlots) * G + cta;
          unsigned long long* r2 = reinterpret_cast<unsigned long long*>(p.qrow + s2 * kQStride);
          for (int i = lane; i < w; i += 32) st_relaxed_u64(r2 + i, kSentinel);
          if (lane < 2) st_relaxed_u64(r2 + kMaxW + lane, kSentinel);
          if (lane == 0) st_relaxed_u64(p.qkey + s2 * kQKeyStride, 0ull);
        }
        // Poll every slot of this step until all keys are present.  Whenever the best key
        // seen so far changes, that candidate's record is fetched at once, so the fetch of
        // the final winner is usually complete when its last competitor's key arrives.
        const unsigned long long* kq = p.qkey + (size_t)q * G * kQKeyStride;
        unsigned long long kv[kPollSlots];
#pragma unroll
        for (int k = 0; k < kPollSlots; ++k) kv[k] = 0ull;
        int pref = -1;                                // slot whose record is in xv, alpha, beta
        unsigned spins = 0;
        while (true) {
          bool mine = true;
          unsigned long long bk = 0ull;
          int bs = -1;
#pragma unroll
          for (int k = 0; k < kPollSlots; ++k) {
            const int s = lane + 32 * k;
            if (s < G) {
              if (kv[k] == 0ull) kv[k] = ld_relaxed_u64(kq + (size_t)s * kQKeyStride);
              if (kv[k] == 0ull) mine = false;
              else if (kv[k] > bk) { bk = kv[k]; bs = s; }
            }
          }
          const Cand b = warp_max_key(Cand{bk, 0, 0, bs});
          const bool all = __all_sync(0xffffffffu, mine);
          if ((b.v >> kPosBits) != 0ull && b.aux != pref) {
            pref = b.aux;
            const double* src = p.qrow + ((size_t)q * G + pref) * kQStride;
#pragma unroll
            for (int k = 0; k < NV; ++k) {
              const int i = lane + 32 * k;
              xv[k] = i < w ? ld_relaxed_f64(src + i) : 0.0;
            }
            alpha = ld_relaxed_f64(src + kMaxW);
            beta = ld_relaxed_f64(src + kMaxW + 1);
          }
          if (all) {
            g = b;
            break;
          }
          // give up (warp-uniformly) after about as long as the other bounded waits, or
          // when another CTA has recorded an error
          const bool stop = ++spins > (limit >> 3) || ((spins & 63) == 0 && dev_status(st) != 0);
          if (__any_sync(0xffffffffu, stop)) {
            if (lane == 0 && atomicCAS(&st->status, 0, PRRP_ERR_TIMEOUT) == 0) st->timeout_site = 1;
            ok = 0;
            break;
          }
        }
        // Exchange fence, once every kQFenceEvery steps.  As a release, it orders this CTA's
        // slot preparations so far before its next key; as an acquire, after every CTA's
        // key of this step, it makes every CTA's preparations released by their previous
        // exchange fence visible.  A slot prepared at step s is released by the first
        // fence at a step >= s and acquired by the next one, at most 2 kQFenceEvery - 1
        // steps later, before its next use at step s + kQSlots - 2.
        if (t % kQFenceEvery == kQFenceEvery - 1) fence_acq_rel_gpu();
        if (ok && (g.v >> kPosBits) != 0ull) {
          // words of the winner's record (its row, alpha, beta) still holding the sentinel
          // are read again
          const double* src = p.qrow + ((size_t)q * G + g.aux) * kQStride;
          unsigned spins2 = 0;
          while (true) {
            bool pending = vbits(alpha) == kSentinel || vbits(beta) == kSentinel;
#pragma unroll
            for (int k = 0; k < NV; ++k)
              if (lane + 32 * k < w && vbits(xv[k]) == kSentinel) pending = true;
            if (!__any_sync(0xffffffffu, pending)) break;
            const bool stop = ++spins2 > (limit >> 3) || ((spins2 & 63) == 0 && dev_status(st) != 0);
            if (__any_sync(0xffffffffu, stop)) {
              if (lane == 0 && atomicCAS(&st->status, 0, PRRP_ERR_TIMEOUT) == 0) st->timeout_site = 5;
              ok = 0;
              break;
            }
#pragma unroll
            for (int k = 0; k < NV; ++k) {
              const int i = lane + 32 * k;
              if (i < w && vbits(xv[k]) == kSentinel) xv[k] = ld_relaxed_f64(src + i);
            }
            if (vbits(alpha) == kSentinel) alpha = ld_relaxed_f64(src + kMaxW);
            if (vbits(beta) == kSentinel) beta = ld_relaxed_f64(src + kMaxW + 1);
          }
        }
      } else {
        const int q = par;
        const unsigned phase = (t >> 1) & 1;
        if (lane < 2) s_ab[q][lane] = vval(kSentinel);
        __syncwarp();
        // push this CTA's key (and its row's local index) into every CTA, then arrive there
        if (lane < G) {
          cl_st_u64(cl_map(&s_rk[q * 16 + cta], lane), has ? d.v : kNoCand);
          cl_st_s32(cl_map(&s_raux[q * 16 + cta], lane), d.aux);
          mbar_arrive_remote(cl_map(&s_mb[q], lane));
        }
        named_arrive(kBarHelp, 64);                   // the helper may fill in alpha, beta
        unsigned spins = 0;
        while (!mbar_try_wait_cluster(&s_mb[q], phase)) {
          if (++spins > (limit >> 3) || ((spins & 63) == 0 && dev_status(st) != 0)) {
            if (atomicCAS(&st->status, 0, PRRP_ERR_TIMEOUT) == 0) st->timeout_site = 3;
            ok = 0;
            break;
          }
        }
        ok = __all_sync(0xffffffffu, ok);
        if (ok) {
          Cand c{0ull, 0, 0, -1};
          if (lane < G) c = Cand{s_rk[q * 16 + lane], 0, 0, lane};
          g = warp_max_key(c);
          if ((g.v >> kPosBits) != 0ull) {
            const int ar = s_raux[q * 16 + g.aux];
#pragma unroll
            for (int k = 0; k < NV; ++k) {
              const int i = lane + 32 * k;
              xv[k] = i < w ? cl_ld_f64(cl_map(&Ps[ar * SP + i], g.aux)) : 0.0;
            }
            const uint32_t ab = cl_map(&s_ab[q][0], g.aux);
            alpha = cl_ld_f64(ab);
            beta = cl_ld_f64(ab + 8u);
            unsigned spins2 = 0;
            while (vbits(alpha) == kSentinel || vbits(beta) == kSentinel) {
              if (++spins2 > (limit >> 3)) {
                if (atomicCAS(&st->status, 0, PRRP_ERR_TIMEOUT) == 0) st->timeout_site = 6;
                ok = 0;
                break;
              }
              alpha = cl_ld_f64(ab);
              beta = cl_ld_f64(ab + 8u);
            }
            ok = __all_sync(0xffffffffu, ok);
          }
        }
      }
      if (ok && key_norm_zero(g.v)) {           // the largest remaining norm is zero: rank < w
        if (cta == 0 && lane == 0) set_error(st, PRRP_ERR_SINGULAR, p.col_offset + t + 1);
        ok = 0;
      }
      if (ok) {
        // the reflector of the winner's row, v = x - alpha e_t; R(0:t, t) and R(t, t)
        double x0 = 0.0;
#pragma unroll
        for (int k = 0; k < NV; ++k)
          if (k == (t >> 5)) x0 = xv[k];
        x0 = __shfl_sync(0xffffffffu, x0, t & 31);
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          const int i = lane + 32 * k;
          if (i < w) {
            s_v[par][i] = (i == t) ? x0 - alpha : xv[k];
            if (i < t) Rs[i * W + t] = xv[k];
          }
        }
        if (lane == 0) {
          Rs[t * W + t] = alpha;
          s_beta[par] = beta;
          s_pw[par] = key_pos(g.v);
        }
      }
      if (lane == 0) {
        s_qok[par] = ok;
        if (!ok) s_abort = 1;
      }
      __syncwarp();
      named_arrive(kBarWin, kThreads);                // the row warps may apply step t
      if (!ok) break;
    }
  } else if (warp == 1) {
    // ---- helper warp: the reflector of this CTA's candidate, off the critical path ----
    for (int t = 0; t < w; ++t) {
      const int par = t & 1;
      named_sync(kBarProp, kThreads);
      Cand d = (lane >= kRowWarp0 && lane < kWarps) ? s_wc[lane] : Cand{0ull, 0, 0, -1};
      d = warp_max_key(d);
      const bool has = d.v > kNoCand && d.aux >= 0;
      double alpha = 0.0, beta = 0.0;
      if (has && lane == 0) reflector(Ps[d.aux * SP + t], nrm[d.aux], &alpha, &beta);
      named_sync(kBarHelp, 64);                       // the record and its sentinels are out
      if (has && lane == 0) {
        if constexpr (!CL) {
          double* rec = p.qrow + ((size_t)(t % kQSlots) * G + cta) * kQStride;
          rec[kMaxW] = alpha;
          rec[kMaxW + 1] = beta;
        } else {
          s_ab[par][0] = alpha;
          s_ab[par][1] = beta;
        }
      }
      __syncwarp();
      named_sync(kBarWin, kThreads);                  // the step's outcome
      if (!s_qok[par]) break;
    }
  } else {
    // ---- row warps ----
    unsigned long long kbest = 0ull;
    int rbest = -1;
    for (int r = wr0 + tw; r < wr1; r += TPW) {
      double s = 0.0;
      for (int i = tl; i < w; i += TEAM) { const double x = Ps[r * SP + i]; s = fma(x, x, s); }
      s = team_sum<TEAM>(s, tmask);
      if (tl == 0) {
        nrm[r] = s;
        thr[r] = 1e-4 * s;
        pos[r] = r0 + r;
        pend[r] = 0;
        // unpivoted QR (CALU_PRRP's L21): the row at position 0 is the only proposal
        const unsigned long long k =
            p.nopivot ? (r0 + r == 0 ? qrcp_key(s, 0) | kTopBit : 0ull) : qrcp_key(s, r0 + r);
        if (k > kbest) { kbest = k; rbest = r; }
      }
    }
    {
      const Cand c = warp_max_key(Cand{kbest, 0, 0, rbest});
      if (lane == 0) s_wc[warp] = c;
    }
    __syncwarp();
    named_arrive(kBarProp, kThreads);
    for (int t = 0; t < w; ++t) {
      const int par = t & 1;
      named_sync(kBarWin, kThreads);                 // the winner of step t and its reflector
      if (!s_qok[par]) break;
      const double* vs = s_v[par];
      const double beta = s_beta[par];
      const int pw = s_pw[par];
      kbest = 0ull;
      rbest = -1;
      // critical part: dot product, new B(t, q), norm downdate, proposal for step t + 1
      for (int r = wr0 + tw; r < wr1; r += TPW) {
        const int pr = pos[r];
        if (pr < t) continue;                           // selected at an earlier step
        if (pr == pw) {                                  // the pivot row: now R(:, t)
          if (tl == 0) pos[r] = t;
          continue;
        }
        double* x = Ps + r * SP;
        double dot;
        if constexpr (TEAM == 1) {
          // four chains cut the dependent-FMA latency of a whole row per lane
          double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
          int i = t;
          for (; i + 3 < w; i += 4) {
            s0 = fma(vs[i], x[i], s0);
            s1 = fma(vs[i + 1], x[i + 1], s1);
            s2 = fma(vs[i + 2], x[i + 2], s2);
            s3 = fma(vs[i + 3], x[i + 3], s3);
          }
          for (; i < w; ++i) s0 = fma(vs[i], x[i], s0);
          dot = (s0 + s1) + (s2 + s3);
        } else {
          double sd0 = 0.0, sd1 = 0.0;    // two chains halve the dependent-FMA latency
          int i = t + tl;
          for (; i + TEAM < w; i += 2 * TEAM) {
            sd0 = fma(vs[i], x[i], sd0);
            sd1 = fma(vs[i + TEAM], x[i + TEAM], sd1);
          }
          if (i < w) sd0 = fma(vs[i], x[i], sd0);
          dot = team_sum<TEAM>(sd0 + sd1, tmask);
        }
        const double f = beta * dot;
        double xt = 0.0;
        if (tl == 0) {
          xt = fma(-f, vs[t], x[t]);
          x[t] = xt;
        }
        xt = __shfl_sync(tmask, xt, lane & ~(TEAM - 1));
        // remaining squared norm for step t+1: downdate, recomputed exactly when it has
        // fallen below 1e-4 of its last exact value (bounds the cancellation error)
        double n2 = fma(-xt, xt, nrm[r]);
        int defer = 1;
        if (!gt_nonneg(n2, thr[r])) {
          for (int i2 = t + tl + (tl == 0 ? TEAM : 0); i2 < w; i2 += TEAM) x[i2] = fma(-f, vs[i2], x[i2]);
          __syncwarp(tmask);
          double e2 = 0.0;
          for (int i2 = t + 1 + tl; i2 < w; i2 += TEAM) e2 = fma(x[i2], x[i2], e2);
          n2 = team_sum<TEAM>(e2, tmask);
          if (tl == 0) thr[r] = 1e-4 * n2;
          defer = 0;
        }
        __syncwarp(tmask);
        if (tl == 0) {
          const int np = (pr == t) ? pw : pr;
          nrm[r] = n2;
          pos[r] = np;
          fpend[r] = f;
          pend[r] = defer;
          const unsigned long long k =
              p.nopivot ? (np == t + 1 ? qrcp_key(n2, np) | kTopBit : 0ull) : qrcp_key(n2, np);
          if (k > kbest) { kbest = k; rbest = r; }
        }
      }
      __syncwarp();
      if (t + 1 < w) {
        const Cand c = warp_max_key(Cand{kbest, 0, 0, rbest});
        // the proposed row's values are published: finish its update first
        if (c.aux >= 0 && pend[c.aux]) {
          const double f = fpend[c.aux];
          double* x = Ps + c.aux * SP;
          for (int i = t + 1 + lane; i < w; i += 32) x[i] = fma(-f, vs[i], x[i]);
          __syncwarp();
          if (lane == 0) pend[c.aux] = 0;
        }
        if (lane == 0) s_wc[warp] = c;
        __syncwarp();
        named_arrive(kBarProp, kThreads);
      }
      // the rest of the step's row updates, while warp 0 exchanges the proposals
      for (int r = wr0 + tw; r < wr1; r += TPW) {
        if (!pend[r]) continue;
        const double f = fpend[r];
        double* x = Ps + r * SP;
        for (int i = t + tl + (tl == 0 ? TEAM : 0); i < w; i += TEAM) x[i] = fma(-f, vs[i], x[i]);
        __syncwarp(tmask);
        if (tl == 0) pend[r] = 0;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  if (s_abort) goto done;

  // ---------------- M = R11^-1 R12 (back substitution) ----------------
  // the diagonal's reciprocals once per CTA (a division is ~8 FP64 instructions)
  for (int i = tid; i < w; i += blockDim.x) rdiag[i] = 1.0 / Rs[i * W + i];
  __syncthreads();
  for (int r = wr0 + tw; r < wr1; r += TPW) {
    if (pos[r] < w) continue;
    double* b = Ps + r * SP;
    for (int i = w - 1; i >= 0; --i) {
      const int owner = i & (TEAM - 1);
      double mi = 0.0;
      if (tl == owner) mi = b[i] * rdiag[i];
      mi = __shfl_sync(tmask, mi, (lane & ~(TEAM - 1)) | owner);
      if (tl == owner) b[i] = mi;
      for (int k = tl; k < i; k += TEAM) b[k] = fma(-Rs[k * W + i], mi, b[k]);
    }
  }

  // ---------------- tau-bounded interchanges ----------------
  {
  int swaps = 0;
  for (int it = 0; !p.nopivot; ++it) {
    const int par = it & 1;
    if (warp >= kRowWarp0) {
      Cand c{0ull, 0x7fffffff, 0x7fffffff, -1};
      for (int r = wr0 + tw; r < wr1; r += TPW) {
        const int pr = pos[r];
        if (pr < w) continue;
        Cand d{0ull, pr - w, 0x7fffffff, r};
        for (int i = tl; i < w; i += TEAM) {
          const unsigned long long a = abs_bits(Ps[r * SP + i]);
          if (a > d.v || d.k2 == 0x7fffffff) { d.v = a; d.k2 = i; }
        }
        if (better(d, c)) c = d;
      }
      c = warp_argmax(c);
      if (lane == 0) s_wc[warp] = c;
    }
    __syncthreads();
    if (warp == 0) {
      // this CTA's best, its record, the exchange, the global winner and its row
      Cand d = (lane >= kRowWarp0 && lane < kWarps) ? s_wc[lane] : Cand{0ull, 0x7fffffff, 0x7fffffff, -1};
      d = warp_argmax(d);
      const bool has = d.v != 0ull && d.aux >= 0;
      const size_t slot = (size_t)par * G + cta;
      double* xv = CL ? &s_xval[par] : p.xval + slot * kXVal;
      double* xr = CL ? s_xrow + par * W : p.xvec + slot * kMaxW;
      if (lane == 0) {
        xv[0] = vval(d.v);
        if (CL) s_xkey[par] = make_int2(d.k1, d.k2);
        else p.xkey[slot] = make_int2(d.k1, d.k2);
      }
      if (has)
        for (int i = lane; i < w; i += 32) xr[i] = Ps[d.aux * SP + i];
      __syncwarp();
      int ok = 1;
      if (lane == 0) {
        const unsigned target = (it + 1) * G;
        unsigned spins = 0;
        if constexpr (CL) {
          const uint32_t ctr = cl_map(&s_ctr, 0);
          cl_fence();
          cl_arrive(ctr);
          while (cl_ld_acquire(ctr) < target) {
            if (++spins > limit) {
              if (atomicCAS(&st->status, 0, PRRP_ERR_TIMEOUT) == 0) st->timeout_site = 4;
              ok = 0;
              break;
            }
            __nanosleep(20);
          }
        } else {
          // release: this warp's record (ordered by the warp barrier above) before the
          // arrival; acquire: the other CTAs' records after the last arrival is seen
          asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&st->barrier) : "memory");
          while (ld_acquire_u32(&st->barrier) < target) {
            if (dev_status(st) != 0) { ok = 0; break; }
            if (++spins > limit) {
              if (atomicCAS(&st->status, 0, PRRP_ERR_TIMEOUT) == 0) st->timeout_site = 2;
              ok = 0;
              break;
            }
            __nanosleep(32);
          }
        }
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (ok) {
        Cand g{0ull, 0x7fffffff, 0x7fffffff, -1};
        if constexpr (CL) {
          // each lane acquires the counter itself (it already holds the target value)
          (void)cl_ld_acquire(cl_map(&s_ctr, 0));
          if (lane < G) {
            const unsigned long long v = vbits(cl_ld_f64(cl_map(&s_xval[par], lane)));
            const int2 k = cl_ld_int2(cl_map(&s_xkey[par], lane));
            g = Cand{v, k.x, k.y, lane};
          }
          g = warp_argmax(g);
          if (g.aux >= 0 && g.v != 0ull) {
            const uint32_t row = cl_map(&s_xrow[par * W], g.aux);
            for (int i = lane; i < w; i += 32) s_v[0][i] = cl_ld_f64(row + 8u * i);
          }
        } else {
          __syncwarp();
          for (int q = lane; q < G; q += 32) {
            const size_t sq = (size_t)par * G + q;
            const int2 k = __ldcg(&p.xkey[sq]);
            const Cand e{vbits(__ldcg(&p.xval[sq * kXVal])), k.x, k.y, q};
            if (better(e, g)) g = e;
          }
          g = warp_argmax(g);
          if (g.aux >= 0 && g.v != 0ull)
            for (int i = lane; i < w; i += 32) s_v[0][i] = __ldcg(&p.xvec[((size_t)par * G + g.aux) * kMaxW + i]);
        }
        if (lane == 0) s_gbest = g;
      }
      if (lane == 0) s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) goto done;

    const Cand g = s_gbest;
    if (g.aux < 0 || !(vval(g.v) > p.tau)) break;   // also ends when there is no remaining row
    if (swaps >= p.max_swaps) {
      if (cta == 0 && tid == 0) set_error(st, PRRP_ERR_SWAP_LIMIT, p.col_offset + 1);
      goto done;
    }
    const int js = g.k1, is = g.k2;
    const double* vs = s_v[0];
    const double mu = vs[is];
    for (int r = wr0 + tw; r < wr1; r += TPW) {
      const int pr = pos[r];
      double* x = Ps + r * SP;
      if (pr == w + js) {                          // enters the selection at slot is
        if (tl == 0) pos[r] = is;
      } else if (pr == is) {                       // leaves the selection to slot js
        for (int k = tl; k < w; k += TEAM) x[k] = (k == is) ? 1.0 / mu : -vs[k] / mu;
        __syncwarp(tmask);
        if (tl == 0) pos[r] = w + js;
      } else if (pr >= w) {
        const int owner = is & (TEAM - 1);
        double f = 0.0;
        if (tl == owner) f = x[is] / mu;
        f = __shfl_sync(tmask, f, (lane & ~(TEAM - 1)) | owner);
        for (int k = tl; k < w; k += TEAM) x[k] = (k == is) ? f : fma(-f, vs[k], x[k]);
      }
    }
    ++swaps;
    __syncthreads();                                // s_v[0] and s_wc are rewritten next
  }

  // ---------------- outputs ----------------
  unsigned long long lmax = 0ull;
  for (int r = wr0 + tw; r < wr1; r += TPW) {
    const int pr = pos[r];
    if (pr < w) continue;
    double* dst = p.L21 + (long long)(pr - w) * p.ldl;
    for (int k = tl; k < w; k += TEAM) {
      const double v = Ps[r * SP + k];
      dst[k] = v;
      lmax = max_bits(lmax, abs_bits(v));
    }
  }
  __syncwarp();
  for (int r = wr0 + lane; r < wr1; r += 32) {
    const int pr = pos[r];
    if (p.order) p.order[pr] = r0 + r;
    if (p.pairs && pr != r0 + r) {
      const unsigned idx = atomicAdd(&st->npairs, 1u);
      p.pairs[2 * idx] = pr;
      p.pairs[2 * idx + 1] = r0 + r;
    }
  }
  for (int off = 16; off > 0; off >>= 1) lmax = max_bits(lmax, __shfl_xor_sync(0xffffffffu, lmax, off));
  if (lane == 0 && warp >= kRowWarp0) atomicMax(&st->l21_bits, lmax);
  if (cta == 0 && tid == 0) {
    st->panel_swaps = swaps;
    st->swaps_total += swaps;
  }
  }
  }
done:
  if constexpr (CL) {
    __syncwarp();
    cl_sync_all();                                  // nobody leaves while others may read its rows
  }
}

template <int W, int TEAM>
static size_t panel_smem_bytes(int rpc) {
  return (size_t)rpc * (W + TEAM) * sizeof(double) + (size_t)W * W * sizeof(double) +
         (size_t)rpc * 3 * sizeof(double) + (size_t)W * sizeof(double) + (size_t)rpc * 2 * sizeof(int) + 16;
}

template <int W, int TEAM>
static cudaError_t launch_panel_wt(PanelParams p, int G, cudaStream_t stream) {
  const size_t smem = panel_smem_bytes<W, TEAM>(p.rows_per_cta);
  cudaError_t e = smem_optin(panel_rrqr_kernel<W, false, TEAM>);
  if (e != cudaSuccess) return e;
  void* args[] = {&p};
  return cudaLaunchCooperativeKernel((const void*)panel_rrqr_kernel<W, false, TEAM>, dim3(G), dim3(kThreads),
                                     args, smem, stream);
}
template <int W>
static cudaError_t launch_panel_w(PanelParams p, int G, cudaStream_t stream) {
  if (p.rows_per_cta >= kManyRows) return launch_panel_wt<W, panel_team(W, true)>(p, G, stream);
  return launch_panel_wt<W, panel_team(W, false)>(p, G, stream);
}

// One cluster of `cs` CTAs (cs up to 16, a non-portable cluster size).
template <int W, int TEAM>
static cudaError_t launch_panel_cluster_wt(PanelParams p, int cs, cudaStream_t stream) {
  const size_t smem = panel_smem_bytes<W, TEAM>(p.rows_per_cta);
  cudaError_t e = smem_optin(panel_rrqr_kernel<W, true, TEAM>);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(panel_rrqr_kernel<W, true, TEAM>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, panel_rrqr_kernel<W, true, TEAM>, p);
}
template <int W>
static cudaError_t launch_panel_cluster_w(PanelParams p, int cs, cudaStream_t stream) {
  if (p.rows_per_cta >= kManyRows) return launch_panel_cluster_wt<W, panel_team(W, true)>(p, cs, stream);
  return launch_panel_cluster_wt<W, panel_team(W, false)>(p, cs, stream);
}

int panel_width_class(int w) { return w <= 16 ? 16 : w <= 32 ? 32 : w <= 64 ? 64 : 128; }

template <int W>
static size_t panel_smem_w(int rpc) {
  return rpc >= kManyRows ? panel_smem_bytes<W, panel_team(W, true)>(rpc)
                          : panel_smem_bytes<W, panel_team(W, false)>(rpc);
}

size_t panel_smem_for(int w, int rpc) {
  switch (panel_width_class(w)) {
    case 16: return panel_smem_w<16>(rpc);
    case 32: return panel_smem_w<32>(rpc);
    case 64: return panel_smem_w<64>(rpc);
    default: return panel_smem_w<128>(rpc);
  }
}

// Panels of at most kClusterRows rows (or PanelParams::cluster_rows, at most
// kClusterRowsMax) run as one thread-block cluster of up to 16 CTAs, 32 rows per CTA up to
// 512 rows and m / 16 beyond (while the CTA's rows fit in shared memory); taller ones as a
// cooperative grid.  For a single factorization the grid is faster once a cluster CTA
// would hold more than 32 rows (each step's FP64 row updates then dominate it), but
// clusters do not serialize across streams, which pays when several factorizations share
// the GPU.
constexpr int kClusterRows = 512;
constexpr int kClusterRowsMax = 4096;

cudaError_t launch_panel(const PanelParams& p, int G, cudaStream_t stream) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (G < 1 || G > kPanelMaxCtas) return cudaErrorInvalidValue;
  const int crows = p.cluster_rows > 0 ? std::min(p.cluster_rows, kClusterRowsMax) : kClusterRows;
  if (p.m <= crows) {
    int cs = 2;
    while (cs < 16 && cs * 32 < p.m) cs *= 2;
    PanelParams q = p;
    q.rows_per_cta = (p.m + cs - 1) / cs;
    switch (panel_width_class(p.w)) {
      case 16: e = launch_panel_cluster_w<16>(q, cs, stream); break;
      case 32: e = launch_panel_cluster_w<32>(q, cs, stream); break;
      case 64: e = launch_panel_cluster_w<64>(q, cs, stream); break;
      default: e = launch_panel_cluster_w<128>(q, cs, stream); break;
    }
    if (e == cudaSuccess) return cudaSuccess;
    cudaGetLastError();                 // a cluster that cannot be placed: use the grid form
  }
  std::lock_guard<std::mutex> lock(g_coop_mu);
  if (!g_coop_done[dev]) {
    e = cudaEventCreateWithFlags(&g_coop_done[dev], cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  e = cudaStreamWaitEvent(stream, g_coop_done[dev], 0);
  if (e != cudaSuccess) return e;
  switch (panel_width_class(p.w)) {
    case 16: e = launch_panel_w<16>(p, G, stream); break;
    case 32: e = launch_panel_w<32>(p, G, stream); break;
    case 64: e = launch_panel_w<64>(p, G, stream); break;
    default: e = launch_panel_w<128>(p, G, stream); break;
  }
  if (e != cudaSuccess) return e;
  return cudaEventRecord(g_coop_done[dev], stream);
}

cudaError_t launch_cooperative_chained(const void* func, int grid, int threads, void** args, size_t smem,
                                       cudaStream_t stream) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_coop_mu);
  if (!g_coop_done[dev]) {
    e = cudaEventCreateWithFlags(&g_coop_done[dev], cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  e = cudaStreamWaitEvent(stream, g_coop_done[dev], 0);
  if (e != cudaSuccess) return e;
  e = cudaLaunchCooperativeKernel(func, dim3(grid), dim3(threads), args, smem, stream);
  if (e != cudaSuccess) return e;
  return cudaEventRecord(g_coop_done[dev], stream);
}

}  // namespace prrp
