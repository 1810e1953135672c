// CALU_PRRP tournament pivoting (Section 3.1): the panel's rows are cut into leaves of
// `leaf` contiguous rows (the last leaf takes the remainder); the strong RRQR of each
// leaf's transpose (Algorithm 2) selects w candidate rows, which lead their leaf; then a
// binary tree merges consecutive nodes, left then right: the node matrix is the left
// node's w candidates followed by the right node's, its strong RRQR selects w rows, and
// its permutation acts on the positions of those 2w rows, so the selected rows take the
// left node's candidate positions.  An unpaired last node goes up unchanged.  The root's
// rows end at positions 0..w-1 of the panel.
//
// One cooperative launch runs the whole tree: every CTA runs whole nodes (one node's strong
// RRQR entirely in its shared memory, at most 255 rows), the nodes of a level in parallel,
// and a bounded grid barrier separates the levels.  Rows are not moved while the tree runs:
// pmap (position -> panel row) is updated node by node and the composed permutation is
// applied to whole rows once afterwards (launch_gather_permute).
//
// The arithmetic of a node is that of the LU_PRRP panel kernel (the same keys, reflector,
// downdating with its recompute guard, back substitution and basis-exchange interchanges,
// selection decided on FP64 values), so the tournament's pivots agree with the oracle's
// wherever its decisions are untied.
//
// The same kernel runs the trees of block parallel and block pairwise LU_PRRP (Section 5,
// Appendix E), one level per launch: there each node also eliminates the rows it does not
// select, with D = (R11^-1 R12)^T written into their panel columns, and
// tree_eliminate_kernel then applies A_e -= D_e A_sel to their trailing columns before the
// next level's selection (which reads only panel columns of rows not yet updated).
#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "select.cuh"

namespace prrp {

using namespace sel;

namespace {

constexpr int kTThreads = 256;
constexpr int kTWarps = kTThreads / 32;
constexpr int kNodeMax = kTreeNodeMaxRows;   // CALU: a leaf < 2 leaf <= 256 rows, a merge 2 w
constexpr int kTTeam = 4;

template <int W>
constexpr size_t tourn_smem_bytes() {
  return (size_t)kNodeMax * (W + kTTeam) * sizeof(double) + (size_t)W * W * sizeof(double) +
         2 * (size_t)kNodeMax * sizeof(double) + (size_t)W * sizeof(double) + 3 * (size_t)kNodeMax * sizeof(int) + 16;
}

// Nodes at level h of the tree, and the panel positions of node `node` (0 rows: the node
// is unpaired and goes up unchanged).  Writes gpos[0..rows) with stride `stride` from
// `first` (so that a CTA's threads can share the work).
__host__ __device__ inline int tree_nodes(const TournParams& p, int h) {
  return p.mode == 2 ? 1 : (p.nleaf + (1 << h) - 1) >> h;
}
__device__ inline int tree_node_rows(const TournParams& p, int h, int node, int* gpos, int first, int stride) {
  const int w = p.w;
  if (p.mode == 2) {                                  // flat tree: block h after positions 0..w-1
    const int r0 = h == 0 ? 0 : h * p.leaf;
    const int r1 = h == p.nleaf - 1 ? p.m : (h + 1) * p.leaf;
    const int lead = h == 0 ? 0 : w;
    const int nr = lead + (r1 - r0);
    for (int k = first; k < nr; k += stride) gpos[k] = k < lead ? k : r0 + (k - lead);
    return nr;
  }
  if (h == 0) {
    const int r0 = node * p.leaf;
    const int r1 = node == p.nleaf - 1 ? p.m : r0 + p.leaf;
    for (int k = first; k < r1 - r0; k += stride) gpos[k] = r0 + k;
    return r1 - r0;
  }
  const int a = node << h, b = a + (1 << (h - 1));
  if (b >= p.nleaf) return 0;
  for (int k = first; k < 2 * w; k += stride) gpos[k] = k < w ? a * p.leaf + k : b * p.leaf + (k - w);
  return 2 * w;
}

template <int W>
__global__ void __launch_bounds__(kTThreads, 1) tournament_kernel(TournParams p) {
  constexpr int TEAM = kTTeam;
  constexpr int TPW = 32 / TEAM;
  constexpr int SP = W + TEAM;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* Ps = reinterpret_cast<double*>(smem_raw);      // kNodeMax x SP node rows
  double* Rs = Ps + (size_t)kNodeMax * SP;                // W x W, R11 of the node
  double* nrm = Rs + W * W;                               // remaining squared norms
  double* thr = nrm + kNodeMax;                           // recompute thresholds
  double* rdiag = thr + kNodeMax;                         // W reciprocals of diag(R11)
  int* pos = reinterpret_cast<int*>(rdiag + W);           // node position of local row r
  int* rid = pos + kNodeMax;                              // panel row held by local row r
  int* gpos = rid + kNodeMax;                             // panel position of node position k
  __shared__ Cand s_wc[kTWarps];
  __shared__ Cand s_best;
  __shared__ double s_v[W];
  __shared__ double s_beta;
  __shared__ int s_pw, s_ok, s_abort;

  DevState* st = p.st;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tl = lane & (TEAM - 1), tw = lane / TEAM;
  const unsigned tmask = ((1u << TEAM) - 1u) << (lane & ~(TEAM - 1));
  const int w = p.w;
  if (tid == 0) s_abort = dev_status(st) != 0;
  __syncthreads();
  if (s_abort) return;
  int swaps_total = 0;

  unsigned long long dmax = 0ull;
  for (int h = p.level0; h < p.level1; ++h) {
    const int cnt = tree_nodes(p, h);
    for (int node = blockIdx.x; node < cnt; node += gridDim.x) {
      const int nr = tree_node_rows(p, h, node, gpos, tid, kTThreads);
      if (nr == 0) continue;                              // unpaired: goes up unchanged
      __syncthreads();
      for (int r = tid; r < nr; r += kTThreads) rid[r] = __ldcg(&p.pmap[gpos[r]]);
      __syncthreads();
      for (int e = tid; e < nr * w; e += kTThreads) {
        const int r = e / w, c = e - r * w;
        Ps[r * SP + c] = p.P[(long long)rid[r] * p.ldp + c];
      }
      __syncthreads();
      const int rpw = ((nr + kTWarps - 1) / kTWarps + TPW - 1) / TPW * TPW;
      const int wr0 = min(nr, warp * rpw), wr1 = min(nr, wr0 + rpw);
      for (int r = wr0 + tw; r < wr1; r += TPW) {
        double s = 0.0;
        for (int i = tl; i < w; i += TEAM) { const double x = Ps[r * SP + i]; s = fma(x, x, s); }
        s = team_sum<TEAM>(s, tmask);
        if (tl == 0) { nrm[r] = s; thr[r] = 1e-4 * s; pos[r] = r; }
      }
      __syncthreads();

      // ---- QR with column pivoting of the node matrix ----
      bool good = true;
      for (int t = 0; t < w && good; ++t) {
        unsigned long long kb = 0ull;
        int rb = -1;
        for (int r = wr0 + lane; r < wr1; r += 32) {
          const int pr = pos[r];
          if (pr >= t) {
            const unsigned long long k = qrcp_key(nrm[r], pr);
            if (k > kb) { kb = k; rb = r; }
          }
        }
        const Cand c = warp_max_key(Cand{kb, 0, 0, rb});
        if (lane == 0) s_wc[warp] = c;
        __syncthreads();
        if (warp == 0) {
          Cand d = lane < kTWarps ? s_wc[lane] : Cand{0ull, 0, 0, -1};
          d = warp_max_key(d);
          if (d.aux < 0 || key_norm_zero(d.v)) {         // the largest remaining norm is zero
            if (lane == 0) {
              set_error(st, PRRP_ERR_SINGULAR, p.col_offset + t + 1);
              s_ok = 0;
            }
          } else {
            const double* x = Ps + d.aux * SP;
            double alpha = 0.0, beta = 0.0;
            if (lane == 0) reflector(x[t], nrm[d.aux], &alpha, &beta);
            alpha = __shfl_sync(0xffffffffu, alpha, 0);
            for (int i = lane; i < w; i += 32) {
              s_v[i] = (i == t) ? x[t] - alpha : x[i];
              if (i < t) Rs[i * W + t] = x[i];
            }
            if (lane == 0) {
              Rs[t * W + t] = alpha;
              s_beta = beta;
              s_pw = key_pos(d.v);
              s_ok = 1;
            }
          }
        }
        __syncthreads();
        if (!s_ok) { good = false; break; }
        const double beta = s_beta;
        const int pw = s_pw;
        for (int r = wr0 + tw; r < wr1; r += TPW) {
          const int pr = pos[r];
          if (pr < t) continue;
          if (pr == pw) {
            if (tl == 0) pos[r] = t;
            continue;
          }
          double* x = Ps + r * SP;
          double sd0 = 0.0, sd1 = 0.0;
          int i = t + tl;
          for (; i + TEAM < w; i += 2 * TEAM) {
            sd0 = fma(s_v[i], x[i], sd0);
            sd1 = fma(s_v[i + TEAM], x[i + TEAM], sd1);
          }
          if (i < w) sd0 = fma(s_v[i], x[i], sd0);
          const double f = beta * team_sum<TEAM>(sd0 + sd1, tmask);
          double xt = 0.0;
          for (int i2 = t + tl; i2 < w; i2 += TEAM) {
            const double y = fma(-f, s_v[i2], x[i2]);
            x[i2] = y;
            if (i2 == t) xt = y;
          }
          xt = __shfl_sync(tmask, xt, lane & ~(TEAM - 1));
          double n2 = fma(-xt, xt, nrm[r]);
          if (!gt_nonneg(n2, thr[r])) {
            double e2 = 0.0;
            for (int i2 = t + 1 + tl; i2 < w; i2 += TEAM) e2 = fma(x[i2], x[i2], e2);
            n2 = team_sum<TEAM>(e2, tmask);
            if (tl == 0) thr[r] = 1e-4 * n2;
          }
          __syncwarp(tmask);
          if (tl == 0) { nrm[r] = n2; pos[r] = (pr == t) ? pw : pr; }
        }
        __syncthreads();
      }

      if (good) {
        // ---- M = R11^-1 R12 for the node's other rows ----
        for (int i = tid; i < w; i += kTThreads) rdiag[i] = 1.0 / Rs[i * W + i];
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
        __syncthreads();
        // ---- tau-bounded interchanges ----
        int swaps = 0;
        while (true) {
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
          __syncthreads();
          if (warp == 0) {
            Cand d = lane < kTWarps ? s_wc[lane] : Cand{0ull, 0x7fffffff, 0x7fffffff, -1};
            d = warp_argmax(d);
            if (lane == 0) s_best = d;
            if (d.aux >= 0)
              for (int i = lane; i < w; i += 32) s_v[i] = Ps[d.aux * SP + i];
          }
          __syncthreads();
          const Cand g = s_best;
          if (g.aux < 0 || !(vval(g.v) > p.tau)) break;
          if (swaps >= p.max_swaps) {
            if (tid == 0) set_error(st, PRRP_ERR_SWAP_LIMIT, p.col_offset + 1);
            good = false;
            break;
          }
          const int js = g.k1, is = g.k2;
          const double mu = s_v[is];
          for (int r = wr0 + tw; r < wr1; r += TPW) {
            const int pr = pos[r];
            double* x = Ps + r * SP;
            if (pr == w + js) {
              if (tl == 0) pos[r] = is;
            } else if (pr == is) {
              for (int k = tl; k < w; k += TEAM) x[k] = (k == is) ? 1.0 / mu : -s_v[k] / mu;
              __syncwarp(tmask);
              if (tl == 0) pos[r] = w + js;
            } else if (pr >= w) {
              const int owner = is & (TEAM - 1);
              double f = 0.0;
              if (tl == owner) f = x[is] / mu;
              f = __shfl_sync(tmask, f, (lane & ~(TEAM - 1)) | owner);
              for (int k = tl; k < w; k += TEAM) x[k] = (k == is) ? f : fma(-f, s_v[k], x[k]);
            }
          }
          ++swaps;
          __syncthreads();
        }
        swaps_total += swaps;
      }
      __syncthreads();
      if (good) {    // the node's rows in their new order: position pos[r] holds local row r
        for (int r = tid; r < nr; r += kTThreads) p.pmap[gpos[pos[r]]] = rid[r];
        if (p.mode != 0)   // block LU_PRRP: D of each eliminated row into its panel columns
          for (int e = tid; e < nr * w; e += kTThreads) {
            const int r = e / w, c = e - r * w;
            if (pos[r] >= w) {
              const double d = Ps[r * SP + c];
              p.Pw[(long long)rid[r] * p.ldp + c] = d;
              dmax = max_bits(dmax, abs_bits(d));
            }
          }
      }
      __syncthreads();
    }
    // the next level reads the positions this one wrote (or learns of an error)
    if (h + 1 < p.level1 && !grid_barrier(st, (h - p.level0 + 1) * gridDim.x, 21)) return;
  }
  for (int off = 16; off > 0; off >>= 1) dmax = max_bits(dmax, __shfl_xor_sync(0xffffffffu, dmax, off));
  if (lane == 0 && dmax) atomicMax(&st->l21_bits, dmax);
  if (tid == 0 && swaps_total) atomicAdd(&st->swaps_total, swaps_total);
}

// Block LU_PRRP eliminations of one level: blockIdx.y = node, blockIdx.x = a tile of 32
// trailing columns; the node's w selected rows' tile is staged in shared memory, the D
// rows of its eliminated rows 32 at a time (33.5 KB of static shared memory at w = 64).
constexpr int kElimCols = 32;
constexpr int kElimRows = 32;
template <int W>
__global__ void __launch_bounds__(256) tree_eliminate_kernel(TournParams p, double* __restrict__ A, long long lda,
                                                             int n, int k0) {
  __shared__ int gpos[kNodeMax];
  __shared__ double S[W][kElimCols + 1];
  __shared__ double Dm[kElimRows][W + 1];
  const DevState* st = p.st;
  if (dev_status(st) != 0) return;
  const int h = p.level0, w = p.w, tid = threadIdx.x;
  const int nr = tree_node_rows(p, h, blockIdx.y, gpos, tid, 256);
  if (nr <= w) return;
  __syncthreads();
  const int c0 = k0 + w + blockIdx.x * kElimCols;
  const int cw = min(kElimCols, n - c0);
  if (cw <= 0) return;
  for (int e = tid; e < w * kElimCols; e += 256) {
    const int k = e / kElimCols, c = e - k * kElimCols;
    S[k][c] = c < cw ? A[(long long)(k0 + __ldcg(&p.pmap[gpos[k]])) * lda + c0 + c] : 0.0;
  }
  unsigned long long cmax = 0ull;
  const int col = tid & (kElimCols - 1), rq = tid / kElimCols;       // 8 row phases
  for (int e0 = w; e0 < nr; e0 += kElimRows) {
    const int ne = min(kElimRows, nr - e0);
    __syncthreads();
    for (int e = tid; e < ne * w; e += 256) {
      const int r = e / w, k = e - r * w;
      Dm[r][k] = A[(long long)(k0 + __ldcg(&p.pmap[gpos[e0 + r]])) * lda + k0 + k];
    }
    __syncthreads();
    if (col < cw)
      for (int r = rq; r < ne; r += 256 / kElimCols) {
        double* a = A + (long long)(k0 + __ldcg(&p.pmap[gpos[e0 + r]])) * lda + c0 + col;
        double acc = *a;
        for (int k = 0; k < w; ++k) acc = fma(-Dm[r][k], S[k][col], acc);
        *a = acc;
        cmax = max_bits(cmax, abs_bits(acc));
      }
  }
  for (int off = 16; off > 0; off >>= 1) cmax = max_bits(cmax, __shfl_xor_sync(0xffffffffu, cmax, off));
  if ((tid & 31) == 0 && cmax) atomicMax(&const_cast<DevState*>(st)->gmax_bits, cmax);
}

template <int W>
cudaError_t launch_tournament_w(const TournParams& p, int num_sms, cudaStream_t s) {
  const size_t smem = tourn_smem_bytes<W>();
  cudaError_t e = smem_optin(tournament_kernel<W>);
  if (e != cudaSuccess) return e;
  int nodes = 0;
  for (int h = p.level0; h < p.level1; ++h) nodes = std::max(nodes, tree_nodes(p, h));
  const int grid = std::max(1, std::min(nodes, num_sms));
  TournParams q = p;
  void* args[] = {&q};
  return launch_cooperative_chained((const void*)tournament_kernel<W>, grid, kTThreads, args, smem, s);
}

// Rows k0 + i (all n columns) and perm[k0 + i] take those at k0 + pmap[i]: a gather into
// tmp, then a copy back (two launches, so every read precedes every write).  One warp
// per row, 16-byte accesses where the row allows them.
__global__ void __launch_bounds__(256) gather_rows_kernel(const double* __restrict__ A, long long lda, int n,
                                                          int k0, int m, const int* __restrict__ pmap,
                                                          const int* __restrict__ perm, double* __restrict__ tmp,
                                                          int* __restrict__ ptmp, const DevState* st) {
  if (dev_status(st) != 0) return;
  const int lane = threadIdx.x & 31;
  for (int i = blockIdx.x * 8 + (threadIdx.x >> 5); i < m; i += gridDim.x * 8) {
    const int src = pmap[i];
    if (src == i) continue;
    const double* a = A + (long long)(k0 + src) * lda;
    double* d = tmp + (long long)i * n;
    for (int c = lane; c < n; c += 32) d[c] = a[c];
    if (lane == 0) ptmp[i] = perm[k0 + src];
  }
}

__global__ void __launch_bounds__(256) scatter_rows_kernel(double* __restrict__ A, long long lda, int n, int k0,
                                                           int m, const int* __restrict__ pmap,
                                                           int* __restrict__ perm, const double* __restrict__ tmp,
                                                           const int* __restrict__ ptmp, const DevState* st) {
  if (dev_status(st) != 0) return;
  const int lane = threadIdx.x & 31;
  for (int i = blockIdx.x * 8 + (threadIdx.x >> 5); i < m; i += gridDim.x * 8) {
    if (pmap[i] == i) continue;
    double* a = A + (long long)(k0 + i) * lda;
    const double* d = tmp + (long long)i * n;
    for (int c = lane; c < n; c += 32) a[c] = d[c];
    if (lane == 0) perm[k0 + i] = ptmp[i];
  }
}

}  // namespace

cudaError_t launch_tournament(const TournParams& p, int num_sms, cudaStream_t s) {
  if (p.w < 1 || p.w > 64 || p.m < p.w || p.nleaf < 1 || p.level0 < 0 || p.level1 <= p.level0)
    return cudaErrorInvalidValue;
  if (p.mode == 0 && (p.leaf < p.w || p.leaf > 128)) return cudaErrorInvalidValue;
  if (p.mode != 0 && p.level1 != p.level0 + 1) return cudaErrorInvalidValue;
  if (p.w <= 16) return launch_tournament_w<16>(p, num_sms, s);
  if (p.w <= 32) return launch_tournament_w<32>(p, num_sms, s);
  return launch_tournament_w<64>(p, num_sms, s);
}

cudaError_t launch_tree_eliminate(const TournParams& p, double* A, long long lda, int n, int k0, int num_sms,
                                  cudaStream_t s) {
  (void)num_sms;
  const int nc = n - k0 - p.w;
  if (nc <= 0) return cudaSuccess;
  const dim3 grid((nc + kElimCols - 1) / kElimCols, tree_nodes(p, p.level0));
  if (p.w <= 16) tree_eliminate_kernel<16><<<grid, 256, 0, s>>>(p, A, lda, n, k0);
  else if (p.w <= 32) tree_eliminate_kernel<32><<<grid, 256, 0, s>>>(p, A, lda, n, k0);
  else tree_eliminate_kernel<64><<<grid, 256, 0, s>>>(p, A, lda, n, k0);
  return cudaGetLastError();
}

cudaError_t launch_gather_permute(double* A, long long lda, int n, int k0, int m, const int* pmap, int* perm,
                                  double* tmp, int* ptmp, DevState* st, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  const int grid = std::min((m + 7) / 8, 152 * 8);
  gather_rows_kernel<<<grid, 256, 0, s>>>(A, lda, n, k0, m, pmap, perm, tmp, ptmp, st);
  scatter_rows_kernel<<<grid, 256, 0, s>>>(A, lda, n, k0, m, pmap, perm, tmp, ptmp, st);
  return cudaGetLastError();
}

}  // namespace prrp
