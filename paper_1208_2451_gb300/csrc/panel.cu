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

__device__ __forceinline__ Cand shfl_cand(const Cand& c, int lane_mask, unsigned mask) {
  Cand o;
  o.v = __shfl_xor_sync(mask, c.v, lane_mask);   // 64-bit shuffle
  o.k1 = __shfl_xor_sync(mask, c.k1, lane_mask);
  o.k2 = __shfl_xor_sync(mask, c.k2, lane_mask);
  o.aux = __shfl_xor_sync(mask, c.aux, lane_mask);
  return o;
}

__device__ __forceinline__ Cand warp_best(Cand c) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    Cand o = shfl_cand(c, off, 0xffffffffu);
    if (better(o, c)) c = o;
  }
  return c;
}

// Sum over the 4 lanes of a row team.  Every lane receives the same bits: the xor
// butterfly adds the same pairs in each lane, only commuted.
__device__ __forceinline__ double team_sum(double s) {
  const unsigned mask = 0xfu << ((threadIdx.x & 31) & ~3);
  s += __shfl_xor_sync(mask, s, 1);
  s += __shfl_xor_sync(mask, s, 2);
  return s;
}

}  // namespace

// Warp-centric layout: warp k of a CTA owns a fixed slice of the CTA's rows for the whole
// kernel, and inside a warp 8 teams of 4 lanes work on one row each.  All per-row state
// (values, remaining squared norm, position) is touched only by its own warp, so a QRCP
// step needs just two block-wide syncs (gathering the warps' proposals, releasing the
// warps after the grid barrier); every warp reduces the G proposals of the tournament on
// its own and keeps its own copy of the winning row.
template <int W>
__global__ void __launch_bounds__(kPanelThreads, 1) panel_rrqr_kernel(PanelParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int SP = W + 4;   // row stride: 4 mod 16 doubles keeps team accesses conflict-light
  constexpr int kWarps = kPanelThreads / 32;
  constexpr int kTeamsPerWarp = 32 / kTeam;
  __shared__ Cand s_wc[kWarps];
  __shared__ int s_ok;

  DevState* st = p.st;
  if (dev_status(st) != 0) return;

  const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int tl = lane & (kTeam - 1), tw = lane / kTeam;          // lane in team, team in warp
  const unsigned tmask = 0xfu << (lane & ~3);
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
  double* nref = nrm + rpc;                               // rpc norms at their last exact value
  int* pos = reinterpret_cast<int*>(nref + rpc);          // rpc current positions
  double* vs = vsw + warp * W;

  unsigned nbar = 0;

  for (int e = tid; e < nr * w; e += blockDim.x) {
    const int r = e / w, c = e - r * w;
    Ps[r * SP + c] = p.P[(long long)(r0 + r) * p.ldp + c];
  }
  __syncthreads();
  for (int r = wr0 + tw; r < wr1; r += kTeamsPerWarp) {
    double s = 0.0;
    for (int i = tl; i < w; i += kTeam) { const double x = Ps[r * SP + i]; s = fma(x, x, s); }
    s = team_sum(s);
    if (tl == 0) { nrm[r] = s; nref[r] = s; pos[r] = r0 + r; }
  }
  __syncwarp();

  // Gather the warps' proposals, publish this CTA's best with its row values, grid barrier.
  // Returns false when the barrier gave up (an error is recorded) and the CTA must return.
  auto publish_and_sync = [&](Cand c, int par, unsigned site) -> bool {
    c = warp_best(c);
    if (lane == 0) s_wc[warp] = c;
    __syncthreads();
    if (warp == 0) {
      Cand d = lane < kWarps ? s_wc[lane] : Cand{0ull, 0x7fffffff, 0x7fffffff, -1};
      d = warp_best(d);
      const size_t slot = (size_t)par * G + cta;
      if (lane == 0) { p.xval[slot] = vval(d.v); p.xkey[slot] = make_int2(d.k1, d.k2); }
      if (d.aux >= 0)
        for (int i = lane; i < w; i += 32) p.xvec[slot * kMaxW + i] = Ps[d.aux * SP + i];
      __syncwarp();
      if (lane == 0) {
        __threadfence();
        atomicAdd(&st->barrier, 1u);
        const unsigned target = (nbar + 1) * G;
        const unsigned limit = st->spin_limit ? st->spin_limit : kSpinLimit;
        unsigned spins = 0;
        int ok = 1;
        while (ld_acquire_u32(&st->barrier) < target) {
          if (dev_status(st) != 0) { ok = 0; break; }
          if (++spins > limit) {
            if (atomicCAS(&st->status, 0, PRRP_ERR_TIMEOUT) == 0) st->timeout_site = site;
            ok = 0;
            break;
          }
          __nanosleep(32);
        }
        __threadfence();
        s_ok = ok;
      }
    }
    __syncthreads();
    ++nbar;
    return s_ok != 0;
  };

  // Every warp: the tournament winner among the G proposals of parity `par`.
  auto global_best = [&](int par) -> Cand {
    Cand g{0ull, 0x7fffffff, 0x7fffffff, -1};
    for (int q = lane; q < G; q += 32) {
      const size_t sq = (size_t)par * G + q;
      const int2 k = __ldcg(&p.xkey[sq]);
      Cand d{vbits(__ldcg(&p.xval[sq])), k.x, k.y, q};
      if (better(d, g)) g = d;
    }
    return warp_best(g);
  };

  // ---------------- QR with column pivoting ----------------
  for (int t = 0; t < w; ++t) {
    const int par = t & 1;
    Cand c{0ull, 0x7fffffff, 0, -1};
    for (int r = wr0 + lane; r < wr1; r += 32) {
      const int pr = pos[r];
      if (pr >= t) {
        Cand d{vbits(fmax(nrm[r], 0.0)), pr, 0, r};
        if (better(d, c)) c = d;
      }
    }
    if (!publish_and_sync(c, par, 1)) return;

    const Cand g = global_best(par);
    if (g.v == 0ull) {            // the largest remaining norm is zero: rank < w
      if (cta == 0 && tid == 0) set_error(st, PRRP_ERR_SINGULAR, p.col_offset + t + 1);
      return;
    }
    const int pw = g.k1;
    for (int i = lane; i < w; i += 32) vs[i] = __ldcg(&p.xvec[((size_t)par * G + g.aux) * kMaxW + i]);
    __syncwarp();
    // Reflector H = I - beta v v^T with H x = alpha e_1 for x = B(t:w, p):
    // ||x|| = sqrt of the winner's remaining squared norm, v = x - alpha e_1,
    // v^T v = 2 ||x|| (||x|| + |x_t|), so beta = 1 / (||x|| (||x|| + |x_t|)).
    const double x0 = vs[t];
    const double normx = sqrt(vval(g.v));
    const double alpha = (x0 >= 0.0) ? -normx : normx;
    const double beta = 1.0 / (normx * (normx + fabs(x0)));
    if (warp == 0) {
      for (int i = lane; i < t; i += 32) Rs[i * W + t] = vs[i];
      if (lane == 0) Rs[t * W + t] = alpha;
    }
    __syncwarp();
    if (lane == 0) vs[t] = x0 - alpha;
    __syncwarp();
    for (int r = wr0 + tw; r < wr1; r += kTeamsPerWarp) {
      const int pr = pos[r];
      if (pr < t) continue;                           // selected at an earlier step
      if (pr == pw) {                                  // the pivot row: now R(:, t)
        if (tl == 0) pos[r] = t;
        continue;
      }
      double* x = Ps + r * SP;
      double sd0 = 0.0, sd1 = 0.0;      // two chains halve the dependent-FMA latency
      int i = t + tl;
      for (; i + kTeam < w; i += 2 * kTeam) {
        sd0 = fma(vs[i], x[i], sd0);
        sd1 = fma(vs[i + kTeam], x[i + kTeam], sd1);
      }
      if (i < w) sd0 = fma(vs[i], x[i], sd0);
      const double sdot = team_sum(sd0 + sd1);
      const double f = beta * sdot;
      double xt = 0.0;
      for (int i = t + tl; i < w; i += kTeam) {
        const double y = fma(-f, vs[i], x[i]);
        x[i] = y;
        if (i == t) xt = y;
      }
      // remaining squared norm for step t+1: downdate, recomputed exactly when it has
      // fallen below 1e-4 of its last exact value (bounds the cancellation error)
      xt = __shfl_sync(tmask, xt, lane & ~3);      // x[t] is handled by team lane 0
      double n2 = fma(-xt, xt, nrm[r]);
      const double ref = nref[r];
      if (!(n2 > 1e-4 * ref)) {
        double e2 = 0.0;
        for (int i = t + 1 + tl; i < w; i += kTeam) e2 = fma(x[i], x[i], e2);
        n2 = team_sum(e2);
        if (tl == 0) nref[r] = n2;
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
  for (int r = wr0 + tw; r < wr1; r += kTeamsPerWarp) {
    if (pos[r] < w) continue;
    double* b = Ps + r * SP;
    for (int i = w - 1; i >= 0; --i) {
      const int owner = i & (kTeam - 1);
      double mi = 0.0;
      if (tl == owner) mi = b[i] * rdiag[i];
      mi = __shfl_sync(tmask, mi, (lane & ~3) | owner);
      if (tl == owner) b[i] = mi;
      for (int k = tl; k < i; k += kTeam) b[k] = fma(-Rs[k * W + i], mi, b[k]);
    }
  }
  __syncthreads();              // rdiag shares memory with the warps' winner rows

  // ---------------- tau-bounded interchanges ----------------
  int swaps = 0;
  for (int it = 0;; ++it) {
    const int par = (w + it) & 1;
    Cand c{0ull, 0x7fffffff, 0x7fffffff, -1};
    for (int r = wr0 + tw; r < wr1; r += kTeamsPerWarp) {
      const int pr = pos[r];
      if (pr < w) continue;
      Cand d{0ull, pr - w, 0x7fffffff, r};
      for (int i = tl; i < w; i += kTeam) {
        const unsigned long long a = abs_bits(Ps[r * SP + i]);
        if (a > d.v || d.k2 == 0x7fffffff) { d.v = a; d.k2 = i; }
      }
      Cand o = shfl_cand(d, 1, tmask);
      if (better(o, d)) d = o;
      o = shfl_cand(d, 2, tmask);
      if (better(o, d)) d = o;
      if (better(d, c)) c = d;
    }
    if (!publish_and_sync(c, par, 2)) return;

    const Cand g = global_best(par);
    if (g.aux < 0 || !(vval(g.v) > p.tau)) break;   // also ends when there is no remaining row
    if (swaps >= p.max_swaps) {
      if (cta == 0 && tid == 0) set_error(st, PRRP_ERR_SWAP_LIMIT, p.col_offset + 1);
      return;
    }
    const int js = g.k1, is = g.k2;
    for (int i = lane; i < w; i += 32) vs[i] = __ldcg(&p.xvec[((size_t)par * G + g.aux) * kMaxW + i]);
    __syncwarp();
    const double mu = vs[is];
    for (int r = wr0 + tw; r < wr1; r += kTeamsPerWarp) {
      const int pr = pos[r];
      double* x = Ps + r * SP;
      if (pr == w + js) {                          // enters the selection at slot is
        if (tl == 0) pos[r] = is;
      } else if (pr == is) {                       // leaves the selection to slot js
        for (int k = tl; k < w; k += kTeam) x[k] = (k == is) ? 1.0 / mu : -vs[k] / mu;
        __syncwarp(tmask);
        if (tl == 0) pos[r] = w + js;
      } else if (pr >= w) {
        const int owner = is & (kTeam - 1);
        double f = 0.0;
        if (tl == owner) f = x[is] / mu;
        f = __shfl_sync(tmask, f, (lane & ~3) | owner);
        for (int k = tl; k < w; k += kTeam) x[k] = (k == is) ? f : fma(-f, vs[k], x[k]);
      }
    }
    ++swaps;
    __syncwarp();
  }

  // ---------------- outputs ----------------
  unsigned long long lmax = 0ull;
  for (int r = wr0 + tw; r < wr1; r += kTeamsPerWarp) {
    const int pr = pos[r];
    if (pr < w) continue;
    double* dst = p.L21 + (long long)(pr - w) * p.ldl;
    for (int k = tl; k < w; k += kTeam) {
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

template <int W>
static size_t panel_smem_bytes(int rpc) {
  return (size_t)rpc * (W + 4) * sizeof(double) + (size_t)W * W * sizeof(double) +
         (size_t)(kPanelThreads / 32) * W * sizeof(double) +
         (size_t)rpc * (2 * sizeof(double) + sizeof(int)) + 16;
}

template <int W>
static cudaError_t launch_panel_w(PanelParams p, int G, cudaStream_t stream) {
  const size_t smem = panel_smem_bytes<W>(p.rows_per_cta);
  cudaError_t e = smem_optin(panel_rrqr_kernel<W>);
  if (e != cudaSuccess) return e;
  void* args[] = {&p};
  return cudaLaunchCooperativeKernel((const void*)panel_rrqr_kernel<W>, dim3(G),
                                     dim3(kPanelThreads), args, smem, stream);
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

cudaError_t launch_panel(const PanelParams& p, int G, cudaStream_t stream) {
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
