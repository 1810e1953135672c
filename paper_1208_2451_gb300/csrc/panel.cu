// Panel factorization of LU_PRRP: strong rank revealing QR of the transposed m x w panel
// (Algorithm 2 of Appendix A, applied as in Algorithm 1, lines 3-4).
//
// One persistent cooperative grid owns the panel: CTA c holds a contiguous chunk of panel
// rows in shared memory for the whole kernel, so the panel is read from HBM once.  In the
// paper's notation B = panel^T, so a panel row is a column of B.
//
// QR with column pivoting, step t:
//   * every CTA proposes its row of largest remaining squared norm ||B(t:w, q)||^2 (ties to
//     the smallest position) together with that row's values;
//   * one grid barrier; every warp of every CTA reduces the G proposals identically (a
//     tournament across CTAs), so all agree on the winner p and build the same Householder
//     reflector from its values, H = I - beta v v^T with H x = alpha e_1,
//     alpha = -sign(x_1) ||x||;
//   * the winner takes position t (the row at position t moves to the winner's position),
//     R(0:t, t) and R(t, t) = alpha are recorded, and every warp applies H to its remaining
//     rows with a team of 4 lanes per row (shuffle reductions).  Remaining norms are
//     downdated, ||B(t+1:w, q)||^2 = ||B(t:w, q)||^2 - B(t, q)^2, and recomputed from the
//     values whenever they fall below 1e-4 of their last exact value, which keeps their
//     relative error near 1e-12.
// Then M = R11^-1 R12 for each remaining row by back substitution.  While the largest
// |M_ij| exceeds tau (ties to the smallest j, then i), selected slot i and remaining row j
// are interchanged; instead of a new QR, M is updated by the exact basis-exchange formulas
// (mu = M_ij, c = M(:, j)):  M'(k, r) = M(k, r) - M(i, r) c_k / mu,  M'(i, r) = M(i, r) / mu,
// and the row leaving the selection gets M'(:, j) = -c / mu with M'(i, j) = 1 / mu.
// Each interchange raises |det R11| by |mu| > tau, so the loop ends (Appendix A).
//
// Outputs: L21 = M^T (row w + r of the final order -> L21 row r), the final position of
// every panel row, and a list of (destination, source) row moves for the permute kernel.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace prrp {

namespace {

// Cooperative panel grids from different streams or contexts must not be resident at the
// same time: two partially resident grids could each wait at their grid barrier for CTAs
// that the other one keeps off the SMs.  Every panel launch on a device therefore waits
// for the previous one (on any stream) through this per-device event chain; other kernels
// still overlap with them freely.
std::mutex g_coop_mu;
cudaEvent_t g_coop_done[64] = {};

// A proposal in an argmax.  The value is a non-negative double (a squared norm or |M_ij|)
// kept as its IEEE bit pattern: for x, y >= 0, x < y exactly when bits(x) < bits(y), so
// the reduction trees compare on the integer pipe instead of the (1/64-rate) FP64 pipe.
struct Cand {
  unsigned long long v;   // bits of the value to maximize (0 with k1 = INT_MAX: none)
  int k1;                 // first tie-break, ascending (position, or remaining slot j)
  int k2;                 // second tie-break, ascending (selected slot i)
  int aux;                // payload: local row index, or proposing CTA
};

__device__ __forceinline__ unsigned long long vbits(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x));
}
__device__ __forceinline__ double vval(unsigned long long b) {
  return __longlong_as_double(static_cast<long long>(b));
}

__device__ __forceinline__ bool better(const Cand& a, const Cand& b) {
  if (a.v != b.v) return a.v > b.v;
  if (a.k1 != b.k1) return a.k1 < b.k1;
  return a.k2 < b.k2;
}

// The best candidate of a full warp (largest value, then smallest k1, then smallest k2),
// returned in every lane: warp-wide max/min reductions on the value's two halves and on
// the tie-breaks, then the payload from the winning lane.
__device__ __forceinline__ Cand warp_argmax(const Cand& c) {
  const unsigned full = 0xffffffffu;
  const unsigned hi = static_cast<unsigned>(c.v >> 32), lo = static_cast<unsigned>(c.v);
  const unsigned mhi = __reduce_max_sync(full, hi);
  const unsigned mlo = __reduce_max_sync(full, hi == mhi ? lo : 0u);
  const bool eq = hi == mhi && lo == mlo;
  const int mk1 = __reduce_min_sync(full, eq ? c.k1 : 0x7fffffff);
  const bool eq1 = eq && c.k1 == mk1;
  const int mk2 = __reduce_min_sync(full, eq1 ? c.k2 : 0x7fffffff);
  const unsigned who = __ballot_sync(full, eq1 && c.k2 == mk2);
  Cand r;
  r.v = (static_cast<unsigned long long>(mhi) << 32) | mlo;
  r.k1 = mk1;
  r.k2 = mk2;
  r.aux = __shfl_sync(full, c.aux, __ffs(who) - 1);
  return r;
}

// QRCP proposals carry one 64-bit key: the squared norm's IEEE bits with the low kPosBits
// bits replaced by (kPosMask - position).  The largest key is the largest norm, ties (and
// norms equal to 2^-32 relative, far inside the 1e-8 decision margin) to the smallest
// position; a key without norm bits (zero norm) still beats "no candidate" (key 0).
constexpr int kPosBits = 20;
constexpr unsigned long long kPosMask = (1ull << kPosBits) - 1;
__device__ __forceinline__ unsigned long long qrcp_key(double nrm, int pos) {
  const long long b = __double_as_longlong(nrm);
  return (static_cast<unsigned long long>(b < 0 ? 0 : b) & ~kPosMask) | (kPosMask - static_cast<unsigned>(pos));
}
__device__ __forceinline__ int key_pos(unsigned long long k) { return static_cast<int>(kPosMask - (k & kPosMask)); }

// The largest key of a full warp with the payload of its lane (keys are unique or zero).
__device__ __forceinline__ Cand warp_max_key(const Cand& c) {
  const unsigned full = 0xffffffffu;
  const unsigned hi = static_cast<unsigned>(c.v >> 32), lo = static_cast<unsigned>(c.v);
  const unsigned mhi = __reduce_max_sync(full, hi);
  const unsigned mlo = __reduce_max_sync(full, hi == mhi ? lo : 0u);
  Cand r;
  r.v = (static_cast<unsigned long long>(mhi) << 32) | mlo;
  r.k1 = 0;
  r.k2 = 0;
  r.aux = __shfl_sync(full, c.aux, __ffs(__ballot_sync(full, c.v == r.v)) - 1);
  return r;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Sum over the TEAM lanes of a row team.  Every lane receives the same bits: the xor
// butterfly adds the same pairs in each lane, only commuted.
template <int TEAM>
__device__ __forceinline__ double team_sum(double s, unsigned tmask) {
#pragma unroll
  for (int off = 1; off < TEAM; off <<= 1) s += __shfl_xor_sync(tmask, s, off);
  return s;
}

// (a > b) for non-negative b: signed compare of the IEEE bit patterns (a negative a, or a
// -0, compares below every positive b; nan above).
__device__ __forceinline__ bool gt_nonneg(double a, double b) {
  return __double_as_longlong(a) > __double_as_longlong(b);
}

// ---- distributed shared memory of a thread-block cluster (cluster mode) ----
__device__ __forceinline__ uint32_t cl_map(const void* p, unsigned rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(r)
               : "r"(static_cast<uint32_t>(__cvta_generic_to_shared(p))), "r"(rank));
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
__device__ __forceinline__ void cl_arrive(uint32_t a) {
  asm volatile("red.release.cluster.shared::cluster.add.u32 [%0], 1;" ::"r"(a) : "memory");
}
__device__ __forceinline__ unsigned cl_ld_acquire(uint32_t a) {
  unsigned v;
  asm volatile("ld.acquire.cluster.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void cl_st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.cluster.shared::cta.u32 [%0], %1;"
               ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(p))), "r"(v) : "memory");
}
__device__ __forceinline__ void cl_fence() { asm volatile("fence.acq_rel.cluster;" ::: "memory"); }
// every thread of every CTA of the cluster (hardware barrier)
__device__ __forceinline__ void cl_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

}  // namespace

// Warp-centric layout: warp k of a CTA owns a fixed slice of the CTA's rows for the whole
// kernel, and inside a warp teams of TEAM = W / 8 lanes work on one row each (8 entries per
// lane at full width).  All per-row state (values, remaining squared norm, position) is
// touched only by its own warp, so a QRCP step needs just two block-wide syncs (gathering
// the warps' proposals, releasing the warps after the grid barrier); every warp reduces
// the G proposals of the tournament on its own and keeps its own copy of the winning row.
// The CTA that proposes a row also computes the reflector of that row (alpha, beta) before
// publishing it, so the square root and division happen once per CTA and step.
//
// CL = false: one cooperative grid; proposals are exchanged through global memory and a
// grid barrier.  CL = true: the grid is one thread-block cluster; every CTA publishes its
// proposal in its own shared memory, a counter in CTA 0 (remote atomics) is the barrier,
// and the proposals and the winning row are read from the other CTAs' shared memory.  The
// cluster's CTAs are co-scheduled by the hardware, so cluster-mode panels from different
// streams may run at the same time.  In cluster mode no CTA leaves before the others are
// done reading its shared memory (a hardware cluster barrier ends the kernel), and every
// decision that ends a loop is taken identically by all CTAs from the same exchanged data.
template <int W, bool CL>
__global__ void __launch_bounds__(kPanelThreads, 1) panel_rrqr_kernel(PanelParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int TEAM = W >= 128 ? 16 : (W >= 64 ? 8 : (W >= 32 ? 4 : 2));
  constexpr int TPW = 32 / TEAM;     // rows per warp pass
  constexpr int SP = W + TEAM;       // row stride: a warp pass touches each bank pair evenly
  constexpr int kWarps = kPanelThreads / 32;
  __shared__ Cand s_wc[kWarps];
  __shared__ int s_ok;
  __shared__ double s_xval[CL ? 2 * kXVal : 1];    // cluster mode: this CTA's records
  __shared__ int2 s_xkey[CL ? 2 : 1];               //   (QRCP: .x = reflector-ready flag)
  __shared__ double s_xrow[CL ? 2 * W : 1];
  __shared__ unsigned s_ctr;                        // cluster mode: the barrier (CTA 0's)
  __shared__ Cand s_gbest;                          // cluster mode: this step's winner,
  __shared__ double s_win[CL ? W : 1];              //   its row and reflector, fetched once
  __shared__ double s_gab[2];                       //   per CTA by warp 0

  DevState* st = p.st;
  if constexpr (!CL) {
    if (dev_status(st) != 0) return;
  } else {
    if (threadIdx.x == 0) {
      s_ctr = 0;
      s_xkey[0] = make_int2(0, 0);
      if (CL) s_xkey[CL ? 1 : 0] = make_int2(0, 0);
    }
    cl_sync_all();                                  // counter and flags zeroed, every CTA running
  }
  {

  const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int tl = lane & (TEAM - 1), tw = lane / TEAM;            // lane in team, team in warp
  const unsigned tmask = (TEAM == 32 ? 0xffffffffu : ((1u << TEAM) - 1u)) << (lane & ~(TEAM - 1));
  const int w = p.w, m = p.m;
  const int rpc = p.rows_per_cta;
  const int r0 = cta * rpc;
  const int nr = max(0, min(rpc, m - r0));
  const int rpw = (nr + kWarps - 1) / kWarps;                   // rows per warp
  const int wr0 = min(nr, warp * rpw), wr1 = min(nr, wr0 + rpw);

  double* Ps = reinterpret_cast<double*>(smem_raw);      // rpc x SP panel rows
  double* Rs = Ps + (size_t)rpc * SP;                     // W x W, R11 (row-major)
  double* vsw = Rs + W * W;                               // kWarps x W: each warp's winner row
  double* nrm = vsw + kWarps * W;                         // rpc remaining squared norms
  double* thr = nrm + rpc;                                // rpc recompute thresholds
  int* pos = reinterpret_cast<int*>(thr + rpc);           // rpc current positions
  double* vs = vsw + warp * W;

  unsigned nbar = 0;

  for (int e = tid; e < nr * w; e += blockDim.x) {
    const int r = e / w, c = e - r * w;
    Ps[r * SP + c] = p.P[(long long)(r0 + r) * p.ldp + c];
  }
  __syncthreads();
  for (int r = wr0 + tw; r < wr1; r += TPW) {
    double s = 0.0;
    for (int i = tl; i < w; i += TEAM) { const double x = Ps[r * SP + i]; s = fma(x, x, s); }
    s = team_sum<TEAM>(s, tmask);
    if (tl == 0) { nrm[r] = s; thr[r] = 1e-4 * s; pos[r] = r0 + r; }
  }
  __syncwarp();

  // Gather the warps' proposals, publish this CTA's best with its row values (and, for a
  // QRCP step t >= 0, the reflector that row would give), grid barrier.  Returns false when
  // the barrier gave up (an error is recorded) and the CTA must return.
  // QRCP steps (t >= 0) exchange packed keys (qrcp_key); the proposing CTA arrives first
  // and computes its row's reflector while the others arrive, publishing alpha and beta
  // behind a ready flag (the exchange's sequence number) that readers wait for.
  auto publish_and_sync = [&](Cand c, int par, unsigned site, int t) -> bool {
    const bool qr = t >= 0;
    c = qr ? warp_max_key(c) : warp_argmax(c);
    if (lane == 0) s_wc[warp] = c;
    __syncthreads();
    if (warp == 0) {
      Cand d = lane < kWarps ? s_wc[lane] : Cand{0ull, 0x7fffffff, 0x7fffffff, -1};
      d = qr ? warp_max_key(d) : warp_argmax(d);
      const size_t slot = (size_t)par * G + cta;
      double* xv = CL ? s_xval + par * kXVal : p.xval + slot * kXVal;
      double* xr = CL ? s_xrow + par * W : p.xvec + slot * kMaxW;
      const bool has = d.v != 0ull && d.aux >= 0;
      if (lane == 0) {
        xv[0] = vval(d.v);
        if (!qr) {
          if (CL) s_xkey[par] = make_int2(d.k1, d.k2);
          else p.xkey[slot] = make_int2(d.k1, d.k2);
        }
      }
      if (has)
        for (int i = lane; i < w; i += 32) xr[i] = Ps[d.aux * SP + i];
      __syncwarp();
      if (lane == 0) {
        const unsigned target = (nbar + 1) * G;
        const unsigned limit = st->spin_limit ? st->spin_limit : kSpinLimit;
        unsigned spins = 0;
        int ok = 1;
        // the reflector of this CTA's candidate, after arriving: H = I - beta v v^T with
        // H x = alpha e_1 for x = B(t:w, row); ||x|| = sqrt of the remaining squared norm,
        // v = x - alpha e_1, v^T v = 2 ||x|| (||x|| + |x_t|)
        auto reflector = [&]() {
          if (qr && has) {
            const double x0 = Ps[d.aux * SP + t];
            const double normx = sqrt(nrm[d.aux]);
            xv[1] = (x0 >= 0.0) ? -normx : normx;
            xv[2] = 1.0 / (normx * (normx + abs_int(x0)));
          }
          if (qr) {
            if (CL) cl_st_release(reinterpret_cast<unsigned*>(&s_xkey[par].x), nbar + 1);
            else st_release_u32(reinterpret_cast<unsigned*>(&p.xkey[slot].x), nbar + 1);
          }
        };
        if constexpr (CL) {
          const uint32_t ctr = cl_map(&s_ctr, 0);
          cl_fence();
          cl_arrive(ctr);
          reflector();
          while (cl_ld_acquire(ctr) < target) {
            if (++spins > limit) {
              if (atomicCAS(&st->status, 0, PRRP_ERR_TIMEOUT) == 0) st->timeout_site = site;
              ok = 0;
              break;
            }
            __nanosleep(20);
          }
        } else {
          // release: this warp's record (ordered by the warp barrier above) before the
          // arrival; acquire: the other CTAs' records after the last arrival is seen
          asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&st->barrier) : "memory");
          reflector();
          while (ld_acquire_u32(&st->barrier) < target) {
            if (dev_status(st) != 0) { ok = 0; break; }
            if (++spins > limit) {
              if (atomicCAS(&st->status, 0, PRRP_ERR_TIMEOUT) == 0) st->timeout_site = site;
              ok = 0;
              break;
            }
            __nanosleep(32);
          }
        }
        s_ok = ok;
      }
      if constexpr (CL) {
        // warp 0 reads the G records once for the whole CTA: each lane acquires the
        // counter itself (it already holds the target value), then the winner's record
        __syncwarp();
        if (s_ok) {
          const uint32_t ctr = cl_map(&s_ctr, 0);
          (void)cl_ld_acquire(ctr);
          Cand g{0ull, 0x7fffffff, 0x7fffffff, -1};
          if (lane < G) {
            const unsigned long long v = vbits(cl_ld_f64(cl_map(&s_xval[par * kXVal], lane)));
            if (qr) {
              g = Cand{v, 0, 0, lane};
            } else {
              const int2 k = cl_ld_int2(cl_map(&s_xkey[par], lane));
              g = Cand{v, k.x, k.y, lane};
            }
          }
          g = qr ? warp_max_key(g) : warp_argmax(g);
          if (g.aux >= 0 && g.v != 0ull) {
            const uint32_t row = cl_map(&s_xrow[par * W], g.aux);
            for (int i = lane; i < w; i += 32) s_win[i] = cl_ld_f64(row + 8u * i);
            if (qr) {
              // the winner's reflector: wait (bounded) for its ready flag
              int ready = 1;
              if (lane == 0) {
                const uint32_t fl = cl_map(&s_xkey[par], g.aux);
                const unsigned limit = st->spin_limit ? st->spin_limit : kSpinLimit;
                unsigned spins = 0;
                while (cl_ld_acquire(fl) != nbar + 1) {
                  if (++spins > limit) {
                    if (atomicCAS(&st->status, 0, PRRP_ERR_TIMEOUT) == 0) st->timeout_site = site + 8;
                    ready = 0;
                    break;
                  }
                }
                if (!ready) s_ok = 0;
              }
              __syncwarp();
              if (lane < 2) s_gab[lane] = cl_ld_f64(cl_map(&s_xval[par * kXVal], g.aux) + 8u * (lane + 1));
            }
          }
          if (lane == 0) s_gbest = g;
        }
      }
    }
    __syncthreads();
    ++nbar;
    return s_ok != 0;
  };

  // Every warp: the tournament winner among the G proposals of parity `par`.
  auto global_best = [&](int par, bool qr) -> Cand {
    if constexpr (CL) {
      return s_gbest;
    } else {
      Cand g{0ull, 0x7fffffff, 0x7fffffff, -1};
      for (int q = lane; q < G; q += 32) {
        const size_t sq = (size_t)par * G + q;
        const unsigned long long v = vbits(__ldcg(&p.xval[sq * kXVal]));
        if (qr) {
          if (v > g.v) g = Cand{v, 0, 0, q};
        } else {
          const int2 k = __ldcg(&p.xkey[sq]);
          Cand d{v, k.x, k.y, q};
          if (better(d, g)) g = d;
        }
      }
      return qr ? warp_max_key(g) : warp_argmax(g);
    }
  };
  // the winning record of parity `par`: row into vs, and (QRCP) alpha, beta
  auto fetch_winner = [&](int par, int q, double* alpha, double* beta) -> bool {
    if constexpr (CL) {
      for (int i = lane; i < w; i += 32) vs[i] = s_win[i];
      if (alpha) {
        *alpha = s_gab[0];
        *beta = s_gab[1];
      }
    } else {
      const size_t gs = (size_t)par * G + q;
      for (int i = lane; i < w; i += 32) vs[i] = __ldcg(&p.xvec[gs * kMaxW + i]);
      if (alpha) {
        // the winner's reflector: wait (bounded) for its ready flag, every lane
        const unsigned limit = st->spin_limit ? st->spin_limit : kSpinLimit;
        unsigned spins = 0;
        bool ready = true;
        while (ld_acquire_u32(reinterpret_cast<const unsigned*>(&p.xkey[gs].x)) != nbar) {
          if (dev_status(st) != 0 || ++spins > limit) {
            if (atomicCAS(&st->status, 0, PRRP_ERR_TIMEOUT) == 0) st->timeout_site = 9;
            ready = false;
            break;
          }
          __nanosleep(16);
        }
        *alpha = __ldcg(&p.xval[gs * kXVal + 1]);
        *beta = __ldcg(&p.xval[gs * kXVal + 2]);
        return __all_sync(0xffffffffu, ready);
      }
    }
    return true;
  };

  // ---------------- QR with column pivoting ----------------
  for (int t = 0; t < w; ++t) {
    const int par = t & 1;
    Cand c{0ull, 0, 0, -1};
    for (int r = wr0 + lane; r < wr1; r += 32) {
      const int pr = pos[r];
      if (pr >= t) {
        const unsigned long long k = qrcp_key(nrm[r], pr);
        if (k > c.v) c = Cand{k, 0, 0, r};
      }
    }
    if (!publish_and_sync(c, par, 1, t)) goto done;

    const Cand g = global_best(par, true);
    if ((g.v >> kPosBits) == 0ull) {  // the largest remaining norm is zero: rank < w
      if (cta == 0 && tid == 0) set_error(st, PRRP_ERR_SINGULAR, p.col_offset + t + 1);
      goto done;
    }
    const int pw = key_pos(g.v);
    double alpha, beta;
    if (!fetch_winner(par, g.aux, &alpha, &beta)) goto done;
    __syncwarp();
    const double x0 = vs[t];
    if (warp == 0) {
      for (int i = lane; i < t; i += 32) Rs[i * W + t] = vs[i];
      if (lane == 0) Rs[t * W + t] = alpha;
    }
    __syncwarp();
    if (lane == 0) vs[t] = x0 - alpha;
    __syncwarp();
    for (int r = wr0 + tw; r < wr1; r += TPW) {
      const int pr = pos[r];
      if (pr < t) continue;                           // selected at an earlier step
      if (pr == pw) {                                  // the pivot row: now R(:, t)
        if (tl == 0) pos[r] = t;
        continue;
      }
      double* x = Ps + r * SP;
      double sd0 = 0.0, sd1 = 0.0;      // two chains halve the dependent-FMA latency
      int i = t + tl;
      for (; i + TEAM < w; i += 2 * TEAM) {
        sd0 = fma(vs[i], x[i], sd0);
        sd1 = fma(vs[i + TEAM], x[i + TEAM], sd1);
      }
      if (i < w) sd0 = fma(vs[i], x[i], sd0);
      const double f = beta * team_sum<TEAM>(sd0 + sd1, tmask);
      double xt = 0.0;
      for (int i = t + tl; i < w; i += TEAM) {
        const double y = fma(-f, vs[i], x[i]);
        x[i] = y;
        if (i == t) xt = y;
      }
      // remaining squared norm for step t+1: downdate, recomputed exactly when it has
      // fallen below 1e-4 of its last exact value (bounds the cancellation error)
      xt = __shfl_sync(tmask, xt, lane & ~(TEAM - 1));      // x[t] is handled by team lane 0
      double n2 = fma(-xt, xt, nrm[r]);
      if (!gt_nonneg(n2, thr[r])) {
        double e2 = 0.0;
        for (int i = t + 1 + tl; i < w; i += TEAM) e2 = fma(x[i], x[i], e2);
        n2 = team_sum<TEAM>(e2, tmask);
        if (tl == 0) thr[r] = 1e-4 * n2;
      }
      __syncwarp(tmask);
      if (tl == 0) { nrm[r] = n2; pos[r] = (pr == t) ? pw : pr; }
    }
    __syncwarp();
  }
  __syncthreads();

  // ---------------- M = R11^-1 R12 (back substitution) ----------------
  // the diagonal's reciprocals once per CTA (a division is ~8 FP64 instructions)
  double* rdiag = vsw;                                    // the winner rows are no longer needed
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
  __syncthreads();              // rdiag shares memory with the warps' winner rows

  // ---------------- tau-bounded interchanges ----------------
  int swaps = 0;
  for (int it = 0;; ++it) {
    const int par = (w + it) & 1;
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
    if (!publish_and_sync(c, par, 2, -1)) goto done;

    const Cand g = global_best(par, false);
    if (g.aux < 0 || !(vval(g.v) > p.tau)) break;   // also ends when there is no remaining row
    if (swaps >= p.max_swaps) {
      if (cta == 0 && tid == 0) set_error(st, PRRP_ERR_SWAP_LIMIT, p.col_offset + 1);
      goto done;
    }
    const int js = g.k1, is = g.k2;
    fetch_winner(par, g.aux, nullptr, nullptr);
    __syncwarp();
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
    __syncwarp();
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
  if (lane == 0) atomicMax(&st->l21_bits, lmax);
  if (cta == 0 && tid == 0) {
    st->panel_swaps = swaps;
    st->swaps_total += swaps;
  }
  }
done:
  if constexpr (CL) {
    __syncwarp();
    cl_sync_all();                                  // nobody leaves while others may read its records
  }
}

template <int W>
static size_t panel_smem_bytes(int rpc) {
  constexpr int TEAM = W >= 128 ? 16 : (W >= 64 ? 8 : (W >= 32 ? 4 : 2));
  return (size_t)rpc * (W + TEAM) * sizeof(double) + (size_t)W * W * sizeof(double) +
         (size_t)(kPanelThreads / 32) * W * sizeof(double) +
         (size_t)rpc * (2 * sizeof(double) + sizeof(int)) + 16;
}

template <int W>
static cudaError_t launch_panel_w(PanelParams p, int G, cudaStream_t stream) {
  const size_t smem = panel_smem_bytes<W>(p.rows_per_cta);
  cudaError_t e = smem_optin(panel_rrqr_kernel<W, false>);
  if (e != cudaSuccess) return e;
  void* args[] = {&p};
  return cudaLaunchCooperativeKernel((const void*)panel_rrqr_kernel<W, false>, dim3(G),
                                     dim3(kPanelThreads), args, smem, stream);
}

// One cluster of `cs` CTAs (cs up to 16, a non-portable cluster size).
template <int W>
static cudaError_t launch_panel_cluster_w(PanelParams p, int cs, cudaStream_t stream) {
  const size_t smem = panel_smem_bytes<W>(p.rows_per_cta);
  cudaError_t e = smem_optin(panel_rrqr_kernel<W, true>);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(panel_rrqr_kernel<W, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(kPanelThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, panel_rrqr_kernel<W, true>, p);
}

int panel_width_class(int w) { return w <= 16 ? 16 : w <= 32 ? 32 : w <= 64 ? 64 : 128; }

size_t panel_smem_for(int w, int rpc) {
  switch (panel_width_class(w)) {
    case 16: return panel_smem_bytes<16>(rpc);
    case 32: return panel_smem_bytes<32>(rpc);
    case 64: return panel_smem_bytes<64>(rpc);
    default: return panel_smem_bytes<128>(rpc);
  }
}

// Panels of at most kClusterRows rows (or PanelParams::cluster_rows, at most
// kClusterRowsMax) run as one thread-block cluster of up to 16 CTAs, 32 rows per CTA up to
// 512 rows and m / 16 beyond (while the CTA's rows fit in shared memory); taller ones as a
// cooperative grid.  For a single
// factorization the grid is faster once a cluster CTA would hold more than 32 rows (each
// step's FP64 row updates then dominate it), but clusters do not serialize across streams,
// which pays when several factorizations share the GPU.
constexpr int kClusterRows = 512;
constexpr int kClusterRowsMax = 4096;

cudaError_t launch_panel(const PanelParams& p, int G, cudaStream_t stream) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
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

}  // namespace prrp
