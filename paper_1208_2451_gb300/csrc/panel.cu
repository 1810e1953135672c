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
//   * one grid barrier; every CTA reduces the G proposals identically (a tournament across
//     CTAs), so all CTAs agree on the winner p and build the same Householder reflector
//     from its values, H = I - beta v v^T with H x = alpha e_1, alpha = -sign(x_1) ||x||;
//   * the winner takes position t (the row at position t moves to the winner's position),
//     R(0:t, t) and R(t, t) = alpha are recorded, and every CTA applies H to its remaining
//     rows with a team of 4 threads per row (shuffle reductions) and recomputes their
//     remaining norms from scratch.
// Then M = R11^-1 R12 for each remaining row by back substitution.  While the largest
// |M_ij| exceeds tau (ties to the smallest j, then i), selected slot i and remaining row j
// are interchanged; instead of a new QR, M is updated by the exact basis-exchange formulas
// (mu = M_ij, c = M(:, j)):  M'(k, r) = M(k, r) - M(i, r) c_k / mu,  M'(i, r) = M(i, r) / mu,
// and the row leaving the selection gets M'(:, j) = -c / mu with M'(i, j) = 1 / mu.
// Each interchange raises |det R11| by |mu| > tau, so the loop ends (Appendix A).
//
// Outputs: L21 = M^T (row w + r of the final order -> L21 row r), the final position of
// every panel row, and a list of (destination, source) row moves for the permute kernel.
#include "common.cuh"
#include "kernels.h"

namespace prrp {

namespace {

struct Cand {
  double v;   // key to maximize (-1 = no candidate)
  int k1;     // first tie-break, ascending (position, or remaining slot j)
  int k2;     // second tie-break, ascending (selected slot i)
  int aux;    // payload: local row index, or proposing CTA
};

__device__ __forceinline__ bool better(const Cand& a, const Cand& b) {
  if (a.v != b.v) return a.v > b.v;
  if (a.k1 != b.k1) return a.k1 < b.k1;
  return a.k2 < b.k2;
}

__device__ __forceinline__ Cand shfl_cand(const Cand& c, int lane_mask, unsigned mask) {
  Cand o;
  o.v = __shfl_xor_sync(mask, c.v, lane_mask);
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

// Block-wide best candidate, returned to every thread.
__device__ Cand block_best(Cand c, Cand* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  c = warp_best(c);
  if (lane == 0) scratch[warp] = c;
  __syncthreads();
  if (warp == 0) {
    Cand d = lane < (int)(blockDim.x >> 5) ? scratch[lane] : Cand{-1.0, 0x7fffffff, 0x7fffffff, -1};
    d = warp_best(d);
    if (lane == 0) scratch[32] = d;
  }
  __syncthreads();
  Cand r = scratch[32];
  __syncthreads();
  return r;
}

// Sum over the 4 lanes of a row team.  Every lane receives the same bits: the xor
// butterfly adds the same pairs in each lane, only commuted.
__device__ __forceinline__ double team_sum(double s) {
  const unsigned mask = 0xfu << ((threadIdx.x & 31) & ~3);
  s += __shfl_xor_sync(mask, s, 1);
  s += __shfl_xor_sync(mask, s, 2);
  return s;
}

__device__ __forceinline__ double warp_sum(double s) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  return s;
}

}  // namespace

template <int W>
__global__ void __launch_bounds__(kPanelThreads, 1) panel_rrqr_kernel(PanelParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int SP = W + 4;   // row stride: 4 mod 16 doubles keeps team accesses conflict-light
  constexpr int kTeams = kPanelThreads / kTeam;
  __shared__ Cand s_red[33];
  __shared__ double s_alpha, s_beta;

  DevState* st = p.st;
  if (dev_status(st) != 0) return;

  const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int tl = tid & (kTeam - 1), team = tid / kTeam;
  const unsigned tmask = 0xfu << (lane & ~3);
  const int w = p.w, m = p.m;
  const int rpc = p.rows_per_cta;
  const int r0 = cta * rpc;
  const int nr = max(0, min(rpc, m - r0));

  double* Ps = reinterpret_cast<double*>(smem_raw);      // rpc x SP panel rows
  double* Rs = Ps + (size_t)rpc * SP;                     // W x W, R11 (row-major)
  double* vs = Rs + W * W;                                // W: broadcast column / reflector
  double* nrm = vs + W;                                   // rpc remaining squared norms
  int* pos = reinterpret_cast<int*>(nrm + rpc);           // rpc current positions

  unsigned nbar = 0;

  for (int e = tid; e < nr * w; e += blockDim.x) {
    const int r = e / w, c = e - r * w;
    Ps[r * SP + c] = p.P[(long long)(r0 + r) * p.ldp + c];
  }
  for (int r = tid; r < nr; r += blockDim.x) pos[r] = r0 + r;
  __syncthreads();
  for (int r = team; r < nr; r += kTeams) {
    double s = 0.0;
    for (int i = tl; i < w; i += kTeam) { const double x = Ps[r * SP + i]; s = fma(x, x, s); }
    s = team_sum(s);
    if (tl == 0) nrm[r] = s;
  }
  __syncthreads();

  // ---------------- QR with column pivoting ----------------
  for (int t = 0; t < w; ++t) {
    const int par = t & 1;
    Cand c{-1.0, 0x7fffffff, 0, -1};
    for (int r = tid; r < nr; r += blockDim.x) {
      const int pr = pos[r];
      if (pr >= t) {
        Cand d{nrm[r], pr, 0, r};
        if (better(d, c)) c = d;
      }
    }
    c = block_best(c, s_red);
    const size_t slot = (size_t)par * G + cta;
    if (tid == 0) { p.xval[slot] = c.v; p.xkey[slot] = make_int2(c.k1, c.k2); }
    if (c.aux >= 0)
      for (int i = tid; i < w; i += blockDim.x) p.xvec[slot * kMaxW + i] = Ps[c.aux * SP + i];
    if (!grid_barrier(st, (++nbar) * G, 1)) return;

    Cand g{-1.0, 0x7fffffff, 0, -1};
    for (int q = tid; q < G; q += blockDim.x) {
      const size_t sq = (size_t)par * G + q;
      const int2 k = __ldcg(&p.xkey[sq]);
      Cand d{__ldcg(&p.xval[sq]), k.x, k.y, q};
      if (better(d, g)) g = d;
    }
    g = block_best(g, s_red);
    if (!(g.v > 0.0)) {           // the largest remaining norm is zero: rank < w
      if (cta == 0 && tid == 0) set_error(st, PRRP_ERR_SINGULAR, p.col_offset + t + 1);
      return;
    }
    const int pw = g.k1;
    for (int i = tid; i < w; i += blockDim.x)
      vs[i] = __ldcg(&p.xvec[((size_t)par * G + g.aux) * kMaxW + i]);
    __syncthreads();
    if (warp == 0) {
      double s = 0.0;
      for (int i = t + lane; i < w; i += 32) s = fma(vs[i], vs[i], s);
      s = warp_sum(s);
      const double x0 = vs[t];
      const double normx = sqrt(s);
      const double alpha = (x0 >= 0.0) ? -normx : normx;
      const double v0 = x0 - alpha;
      double s2 = 0.0;
      for (int i = t + 1 + lane; i < w; i += 32) s2 = fma(vs[i], vs[i], s2);
      s2 = warp_sum(s2);
      const double vv = fma(v0, v0, s2);
      for (int i = lane; i < t; i += 32) Rs[i * W + t] = vs[i];
      __syncwarp();
      if (lane == 0) {
        Rs[t * W + t] = alpha;
        s_alpha = alpha;
        s_beta = (vv == 0.0) ? 0.0 : 2.0 / vv;
        vs[t] = v0;
      }
    }
    __syncthreads();
    const double beta = s_beta;
    for (int r = team; r < nr; r += kTeams) {
      const int pr = pos[r];
      if (pr < t) continue;                           // selected at an earlier step
      if (pr == pw) {                                  // the pivot row: now R(:, t)
        if (tl == 0) pos[r] = t;
        continue;
      }
      const int npos = (pr == t) ? pw : pr;
      double s = 0.0;
      for (int i = t + tl; i < w; i += kTeam) s = fma(vs[i], Ps[r * SP + i], s);
      s = team_sum(s);
      const double f = beta * s;
      double n2 = 0.0;
      for (int i = t + tl; i < w; i += kTeam) {
        const double x = fma(-f, vs[i], Ps[r * SP + i]);
        Ps[r * SP + i] = x;
        if (i > t) n2 = fma(x, x, n2);
      }
      n2 = team_sum(n2);
      if (tl == 0) { nrm[r] = n2; pos[r] = npos; }
    }
    __syncthreads();
  }

  // ---------------- M = R11^-1 R12 (back substitution) ----------------
  for (int r = team; r < nr; r += kTeams) {
    if (pos[r] < w) continue;
    double* b = Ps + r * SP;
    for (int i = w - 1; i >= 0; --i) {
      const int owner = i & (kTeam - 1);
      double mi = 0.0;
      if (tl == owner) mi = b[i] / Rs[i * W + i];
      mi = __shfl_sync(tmask, mi, (lane & ~3) | owner);
      if (tl == owner) b[i] = mi;
      for (int k = tl; k < i; k += kTeam) b[k] = fma(-Rs[k * W + i], mi, b[k]);
    }
  }
  __syncthreads();

  // ---------------- tau-bounded interchanges ----------------
  int swaps = 0;
  for (int it = 0;; ++it) {
    const int par = (w + it) & 1;
    Cand c{-1.0, 0x7fffffff, 0x7fffffff, -1};
    for (int r = team; r < nr; r += kTeams) {
      const int pr = pos[r];
      if (pr < w) continue;
      Cand d{-1.0, pr - w, 0x7fffffff, r};
      for (int i = tl; i < w; i += kTeam) {
        const double a = fabs(Ps[r * SP + i]);
        if (a > d.v) { d.v = a; d.k2 = i; }
      }
      // reduce over the team (same row, so k1 equal): larger |M|, then smaller i
      Cand o = shfl_cand(d, 1, tmask);
      if (better(o, d)) d = o;
      o = shfl_cand(d, 2, tmask);
      if (better(o, d)) d = o;
      if (better(d, c)) c = d;
    }
    c = block_best(c, s_red);
    const size_t slot = (size_t)par * G + cta;
    if (tid == 0) { p.xval[slot] = c.v; p.xkey[slot] = make_int2(c.k1, c.k2); }
    if (c.aux >= 0)
      for (int i = tid; i < w; i += blockDim.x) p.xvec[slot * kMaxW + i] = Ps[c.aux * SP + i];
    if (!grid_barrier(st, (++nbar) * G, 2)) return;

    Cand g{-1.0, 0x7fffffff, 0x7fffffff, -1};
    for (int q = tid; q < G; q += blockDim.x) {
      const size_t sq = (size_t)par * G + q;
      const int2 k = __ldcg(&p.xkey[sq]);
      Cand d{__ldcg(&p.xval[sq]), k.x, k.y, q};
      if (better(d, g)) g = d;
    }
    g = block_best(g, s_red);
    if (!(g.v > p.tau)) break;                  // also ends when there is no remaining row
    if (swaps >= p.max_swaps) {
      if (cta == 0 && tid == 0) set_error(st, PRRP_ERR_SWAP_LIMIT, p.col_offset + 1);
      return;
    }
    const int js = g.k1, is = g.k2;
    for (int i = tid; i < w; i += blockDim.x)
      vs[i] = __ldcg(&p.xvec[((size_t)par * G + g.aux) * kMaxW + i]);
    __syncthreads();
    const double mu = vs[is];
    for (int r = team; r < nr; r += kTeams) {
      const int pr = pos[r];
      double* x = Ps + r * SP;
      if (pr == w + js) {                          // enters the selection at slot is
        if (tl == 0) pos[r] = is;
      } else if (pr == is) {                       // leaves the selection to slot js
        for (int k = tl; k < w; k += kTeam) x[k] = (k == is) ? 1.0 / mu : -vs[k] / mu;
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
    __syncthreads();
  }

  // ---------------- outputs ----------------
  double lmax = 0.0;
  for (int r = team; r < nr; r += kTeams) {
    const int pr = pos[r];
    if (pr < w) continue;
    double* dst = p.L21 + (long long)(pr - w) * p.ldl;
    for (int k = tl; k < w; k += kTeam) {
      const double v = Ps[r * SP + k];
      dst[k] = v;
      lmax = fmax(lmax, fabs(v));
    }
  }
  for (int r = tid; r < nr; r += blockDim.x) {
    const int pr = pos[r];
    if (p.order) p.order[pr] = r0 + r;
    if (p.pairs && pr != r0 + r) {
      const unsigned idx = atomicAdd(&st->npairs, 1u);
      p.pairs[2 * idx] = pr;
      p.pairs[2 * idx + 1] = r0 + r;
    }
  }
  for (int off = 16; off > 0; off >>= 1) lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, off));
  if (lane == 0) atomic_max_nonneg(&st->l21_bits, lmax);
  if (cta == 0 && tid == 0) {
    st->panel_swaps = swaps;
    st->swaps_total += swaps;
  }
}

template <int W>
static size_t panel_smem_bytes(int rpc) {
  return (size_t)rpc * (W + 4) * sizeof(double) + (size_t)W * W * sizeof(double) +
         (size_t)W * sizeof(double) + (size_t)rpc * (sizeof(double) + sizeof(int)) + 16;
}

template <int W>
static cudaError_t launch_panel_w(PanelParams p, int G, cudaStream_t stream) {
  const size_t smem = panel_smem_bytes<W>(p.rows_per_cta);
  cudaError_t e = cudaFuncSetAttribute(panel_rrqr_kernel<W>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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
  switch (panel_width_class(p.w)) {
    case 16: return launch_panel_w<16>(p, G, stream);
    case 32: return launch_panel_w<32>(p, G, stream);
    case 64: return launch_panel_w<64>(p, G, stream);
    default: return launch_panel_w<128>(p, G, stream);
  }
}

}  // namespace prrp
