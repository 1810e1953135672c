// LU_PRRP kernels after the panel (Algorithm 1, lines 5-11), plain FP64.
//
//  scan       max |a_ij| of the input (denominator of g_W, Section 2.2) and NaN/Inf check.
//  permute    Pi_j^T applied to whole rows (line 5): the (destination, source) row moves of
//             the panel are staged through shared memory one column slice per CTA, so all
//             reads of a slice finish before its writes and no grid-wide sync is needed.
//  gemm_fp64  A22 -= L21 A12 (eq. "update", line 7) on the FP64 FMA pipe; tracks max |A22|
//             for the growth factor.
//  diag_gepp  GEPP on the w x w diagonal block (line 10), one CTA.
//  u12        block-row interchanges of GEPP across all other columns and
//             U12 = L11^-1 Pi_jj^T A12 (line 11).
//  lfix       the rows below the block get their final multipliers L21 Pi_jj L11, so the
//             stored factors are the ordinary P A = L U.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace prrp {

// ---------------------------------------------------------------- scan
__global__ void __launch_bounds__(256) scan_kernel(const double* __restrict__ A, long long lda,
                                                   int n, DevState* st) {
  unsigned long long mx = 0ull;                   // max |a| as an IEEE bit pattern
  for (long long row = blockIdx.x; row < n; row += gridDim.x) {
    const double* a = A + row * lda;
    for (int c = threadIdx.x; c < n; c += blockDim.x) mx = max_bits(mx, abs_bits(a[c]));
  }
  for (int off = 16; off > 0; off >>= 1) mx = max_bits(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  const bool bad = mx >= kInfBits;                // an inf or nan somewhere (nan sorts above inf)
  if ((threadIdx.x & 31) == 0) {
    if (!bad) {
      atomicMax(&st->amax_bits, mx);
      atomicMax(&st->gmax_bits, mx);
    }
    if (bad) {
      st->nonfinite = 1;
      set_error(st, PRRP_ERR_NONFINITE);
    }
  }
}

cudaError_t launch_scan(const double* A, long long lda, int n, DevState* st, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int grid = std::min(n, 152 * 8);
  scan_kernel<<<grid, 256, 0, s>>>(A, lda, n, st);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- helpers
__global__ void iota_kernel(int* p, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = i;
}

cudaError_t launch_iota(int* p, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  iota_kernel<<<std::min((n + 255) / 256, 1024), 256, 0, s>>>(p, n);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- permute
constexpr int kPermCols = 32;

__global__ void __launch_bounds__(256) permute_kernel(double* __restrict__ A, long long lda,
                                                      int n, int k0, const int* __restrict__ pairs,
                                                      int max_pairs, int* __restrict__ perm,
                                                      DevState* st) {
  if (dev_status(st) != 0) return;
  extern __shared__ double buf[];                 // max_pairs x kPermCols
  const int np = min((int)st->npairs, max_pairs);
  if (np == 0) return;
  const int c0 = blockIdx.x * kPermCols;
  const int cw = min(kPermCols, n - c0);
  for (int e = threadIdx.x; e < np * cw; e += blockDim.x) {
    const int q = e / cw, c = e - q * cw;
    buf[q * kPermCols + c] = A[(long long)(k0 + pairs[2 * q + 1]) * lda + c0 + c];
  }
  int* pbuf = reinterpret_cast<int*>(buf + (size_t)max_pairs * kPermCols);
  if (blockIdx.x == 0)
    for (int q = threadIdx.x; q < np; q += blockDim.x) pbuf[q] = perm[k0 + pairs[2 * q + 1]];
  __syncthreads();
  for (int e = threadIdx.x; e < np * cw; e += blockDim.x) {
    const int q = e / cw, c = e - q * cw;
    A[(long long)(k0 + pairs[2 * q]) * lda + c0 + c] = buf[q * kPermCols + c];
  }
  if (blockIdx.x == 0)
    for (int q = threadIdx.x; q < np; q += blockDim.x) perm[k0 + pairs[2 * q]] = pbuf[q];
}

cudaError_t launch_permute(double* A, long long lda, int n, int k0, const int* pairs,
                           int max_pairs, int* perm, DevState* st, cudaStream_t s) {
  const size_t smem = (size_t)max_pairs * kPermCols * sizeof(double) + (size_t)max_pairs * sizeof(int);
  cudaError_t e = smem_optin(permute_kernel);
  if (e != cudaSuccess) return e;
  const int grid = (n + kPermCols - 1) / kPermCols;
  permute_kernel<<<grid, 256, smem, s>>>(A, lda, n, k0, pairs, max_pairs, perm, st);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- FP64 Schur update
// C -= L U with a BM x BN tile per CTA (persistent tile loop), 256 threads each owning a
// (BM/16) x (BN/16) register block.  Tiles are taken in order from a counter (one atomic
// per tile, claimed a tile ahead) when one is given, so SMs that also host other kernels
// of the look-ahead simply take fewer tiles; otherwise CTA c takes tiles c, c + grid, ...  The k dimension (<= 128) is staged through
// shared memory in chunks of 64; operands are stored k-major so each thread's row and column
// fragments are contiguous.  The FP64 pipe is the bound: a 128 x 128 x 64 tile is 1M DFMA
// against 128 KB of operand traffic.
constexpr int kGemmKC = 64;

template <int BM, int BN>
__global__ void __launch_bounds__(256, 1) gemm_fp64_kernel(int M, int N, int K,
                                                           const double* __restrict__ L, long long ldl,
                                                           const double* __restrict__ U, long long ldu,
                                                           double* __restrict__ C, long long ldc,
                                                           DevState* st, int track,
                                                           unsigned* __restrict__ tile_ctr) {
  constexpr int TM = BM / 16, TN = BN / 16;
  constexpr int BMP = BM + 2;                      // padded k-major strides
  constexpr int BNP = BN + 2;
  extern __shared__ double sm[];
  double* As = sm;                                 // [kGemmKC][BMP]
  double* Bs = sm + kGemmKC * BMP;                 // [kGemmKC][BNP]
  if (dev_status(st) != 0) return;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int tiles_n = (N + BN - 1) / BN;
  const int tiles = ((M + BM - 1) / BM) * tiles_n;
  unsigned long long cmax = 0ull;               // max |C| as an IEEE bit pattern
  __shared__ int s_tile;
  int tile = blockIdx.x;
  if (tile_ctr) {
    if (tid == 0) s_tile = static_cast<int>(atomicAdd(tile_ctr, 1u));
    __syncthreads();
    tile = s_tile;
  }
  while (tile < tiles) {
    unsigned claim = 0;
    if (tile_ctr && tid == 0) claim = atomicAdd(tile_ctr, 1u);   // consumed after the tile
    const int bm = (tile / tiles_n) * BM, bn = (tile % tiles_n) * BN;
    // warm L2 with this tile's C rows while the operands are staged
    for (int r = tid; r < BM; r += 256)
      if (bm + r < M)
        for (int c = 0; c < BN && bn + c < N; c += 16)
          asm volatile("prefetch.global.L2 [%0];" ::"l"(C + (long long)(bm + r) * ldc + bn + c));
    double acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < K; k0 += kGemmKC) {
      const int kc = min(kGemmKC, K - k0);
      __syncthreads();
      for (int e = tid; e < BM * kGemmKC; e += 256) {
        const int r = e / kGemmKC, k = e - r * kGemmKC;
        double v = 0.0;
        if (bm + r < M && k < kc) v = L[(long long)(bm + r) * ldl + k0 + k];
        As[k * BMP + r] = v;
      }
      for (int e = tid; e < kGemmKC * BN; e += 256) {
        const int k = e / BN, c = e - k * BN;
        double v = 0.0;
        if (bn + c < N && k < kc) v = U[(long long)(k0 + k) * ldu + bn + c];
        Bs[k * BNP + c] = v;
      }
      __syncthreads();
#pragma unroll 2
      for (int k = 0; k < kc; ++k) {
        double a[TM], b[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = As[k * BMP + ty * TM + i];
#pragma unroll
        for (int j = 0; j < TN; ++j) b[j] = Bs[k * BNP + tx * TN + j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int r = bm + ty * TM + i;
      if (r >= M) continue;
      double* crow = C + (long long)r * ldc + bn + tx * TN;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        if (bn + tx * TN + j < N) {
          const double v = crow[j] - acc[i][j];
          crow[j] = v;
          cmax = max_bits(cmax, abs_bits(v));
        }
      }
    }
    if (tile_ctr) {
      __syncthreads();                  // everyone has read the previous s_tile
      if (tid == 0) s_tile = static_cast<int>(claim);
      __syncthreads();
      tile = s_tile;
    } else {
      tile += gridDim.x;
    }
  }
  if (track) {
    for (int off = 16; off > 0; off >>= 1) cmax = max_bits(cmax, __shfl_xor_sync(0xffffffffu, cmax, off));
    if ((tid & 31) == 0) atomicMax(&st->gmax_bits, cmax);
  }
}

template <int BM, int BN>
static cudaError_t launch_gemm_tile(int m, int n, int k, const double* L, long long ldl,
                                    const double* U, long long ldu, double* C, long long ldc,
                                    DevState* st, int track, int grid, cudaStream_t s,
                                    unsigned* tile_ctr = nullptr) {
  const size_t smem = (size_t)kGemmKC * ((BM + 2) + (BN + 2)) * sizeof(double);
  cudaError_t e = smem_optin(gemm_fp64_kernel<BM, BN>);
  if (e != cudaSuccess) return e;
  if (tile_ctr && (e = cudaMemsetAsync(tile_ctr, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
  gemm_fp64_kernel<BM, BN><<<grid, 256, smem, s>>>(m, n, k, L, ldl, U, ldu, C, ldc, st, track, tile_ctr);
  return cudaGetLastError();
}

cudaError_t launch_gemm_fp64(int m, int n, int k, const double* L, long long ldl,
                             const double* U, long long ldu, double* C, long long ldc,
                             DevState* st, int track, int num_sms, cudaStream_t s, int one_per_sm,
                             unsigned* tile_ctr) {
  if (m <= 0 || n <= 0 || k <= 0) return cudaSuccess;
  if (one_per_sm) {
    // leave room on every SM for a co-resident panel CTA (look-ahead): 64 x 64 tiles,
    // one persistent CTA per SM, tiles claimed from tile_ctr when given
    const long long t64 = (long long)((m + 63) / 64) * ((n + 63) / 64);
    return launch_gemm_tile<64, 64>(m, n, k, L, ldl, U, ldu, C, ldc, st, track,
                                    (int)std::min<long long>(t64, num_sms), s, tile_ctr);
  }
  // pick the tile whose wave count wastes least: cost ~ ceil(tiles / sms) * tile area
  const long long t128 = (long long)((m + 127) / 128) * ((n + 127) / 128);
  const long long t64 = (long long)((m + 63) / 64) * ((n + 63) / 64);
  const long long waves128 = (t128 + num_sms - 1) / num_sms;
  const long long waves64 = (t64 + 2 * num_sms - 1) / (2 * num_sms);   // two 64x64 CTAs per SM
  if (waves128 * 4 <= waves64 * 1 + 1 && t128 >= num_sms / 2)
    return launch_gemm_tile<128, 128>(m, n, k, L, ldl, U, ldu, C, ldc, st, track,
                                      (int)std::min<long long>(t128, num_sms), s);
  return launch_gemm_tile<64, 64>(m, n, k, L, ldl, U, ldu, C, ldc, st, track,
                                  (int)std::min<long long>(t64, 2LL * num_sms), s);
}

// ---------------------------------------------------------------- diagonal GEPP
// One CTA; thread (i, q) = (tid / 4, tid % 4) owns row i's columns j = q mod 4.  Per step:
// the pivot search compares |a| by IEEE bit pattern (integer pipe), the pivot row is
// swapped by its owners, and one fused pass forms l_i = a_it / a_tt (one reciprocal per
// step) and a_ij -= l_i a_tj.  w <= 64 rows per pass of 64 row-teams; larger w loops.
__global__ void __launch_bounds__(256) diag_gepp_kernel(double* __restrict__ A, long long lda,
                                                        int k0, int w, int* __restrict__ ipiv,
                                                        int* __restrict__ perm, DevState* st) {
  if (dev_status(st) != 0) return;
  extern __shared__ double D[];                    // w x (w + 1)
  const int WP = w + 1;
  __shared__ int s_p;
  __shared__ unsigned long long s_wv[8];
  __shared__ int s_wi[8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int q = tid & 3, ri = tid >> 2;           // column class, row team
  for (int e = tid; e < w * w; e += blockDim.x) {
    const int i = e / w, j = e - i * w;
    D[i * WP + j] = A[(long long)(k0 + i) * lda + k0 + j];
  }
  __syncthreads();
  for (int t = 0; t < w; ++t) {
    // pivot: first row i >= t of largest |a_it|
    unsigned long long bv = 0ull;
    int bi = 0x7fffffff;
    for (int i = t + tid; i < w; i += blockDim.x) {
      const unsigned long long v = abs_bits(D[i * WP + t]);
      if (v > bv || bi == 0x7fffffff) { bv = v; bi = i; }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long ov = __shfl_xor_sync(0xffffffffu, bv, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { s_wv[warp] = bv; s_wi[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      unsigned long long v = s_wv[0];
      int i0 = s_wi[0];
      for (int k = 1; k < 8; ++k)
        if (s_wv[k] > v || (s_wv[k] == v && s_wi[k] < i0)) { v = s_wv[k]; i0 = s_wi[k]; }
      s_p = (v == 0ull) ? -1 : i0;
      ipiv[t] = i0;
    }
    __syncthreads();
    const int p = s_p;
    if (p < 0) {
      if (tid == 0) set_error(st, PRRP_ERR_SINGULAR, k0 + t + 1);
      return;
    }
    if (p != t)
      for (int j = tid; j < w; j += blockDim.x) {
        const double x = D[t * WP + j];
        D[t * WP + j] = D[p * WP + j];
        D[p * WP + j] = x;
      }
    __syncthreads();
    const double rp = 1.0 / D[t * WP + t];
    const unsigned team_mask = 0xfu << (lane & ~3);
    for (int i = t + 1 + ri; i < w; i += 64) {        // the 4 lanes of a team share i
      const double l = D[i * WP + t] * rp;
      for (int j = t + 1 + q; j < w; j += 4) D[i * WP + j] = fma(-l, D[t * WP + j], D[i * WP + j]);
      __syncwarp(team_mask);                            // all four have read a_it
      if (q == 0) D[i * WP + t] = l;
    }
    __syncthreads();
  }
  unsigned long long umax = 0ull;
  for (int e = tid; e < w * w; e += blockDim.x) {
    const int i = e / w, j = e - i * w;
    const double v = D[i * WP + j];
    A[(long long)(k0 + i) * lda + k0 + j] = v;
    if (j >= i) umax = max_bits(umax, abs_bits(v));
  }
  for (int off = 16; off > 0; off >>= 1) umax = max_bits(umax, __shfl_xor_sync(0xffffffffu, umax, off));
  if (lane == 0) atomicMax(&st->umax_bits, umax);
  if (tid == 0)
    for (int t = 0; t < w; ++t) {
      const int p = ipiv[t];
      if (p != t) {
        const int x = perm[k0 + t];
        perm[k0 + t] = perm[k0 + p];
        perm[k0 + p] = x;
      }
    }
}

cudaError_t launch_diag_gepp(double* A, long long lda, int k0, int w, int* ipiv, int* perm,
                             DevState* st, cudaStream_t s) {
  const size_t smem = (size_t)w * (w + 1) * sizeof(double);
  cudaError_t e = smem_optin(diag_gepp_kernel);
  if (e != cudaSuccess) return e;
  diag_gepp_kernel<<<1, 256, smem, s>>>(A, lda, k0, w, ipiv, perm, st);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- U12 and block-row swaps
constexpr int kU12Cols = 32;

__global__ void __launch_bounds__(kU12Cols) u12_kernel(double* __restrict__ A, long long lda, int n,
                                                       int k0, int w, const int* __restrict__ ipiv,
                                                       int left_slices, int solve, DevState* st) {
  if (dev_status(st) != 0) return;
  extern __shared__ double sh[];
  double* Ls = sh;                                  // w x w (L11, unit lower)
  double* X = sh + w * w;                           // w x kU12Cols
  __shared__ int piv[kMaxW];
  const int tid = threadIdx.x;
  const bool side = blockIdx.x >= left_slices;      // right of the block
  const bool right = side && solve;                 // interchanges and the triangular solve
  const int c0 = side ? k0 + w + (blockIdx.x - left_slices) * kU12Cols : blockIdx.x * kU12Cols;
  const int cend = side ? n : k0;
  const int cw = min(kU12Cols, cend - c0);
  for (int t = tid; t < w; t += blockDim.x) piv[t] = ipiv[t];
  if (right)
    for (int e = tid; e < w * w; e += blockDim.x) {
      const int i = e / w, j = e - i * w;
      Ls[e] = (j < i) ? A[(long long)(k0 + i) * lda + k0 + j] : 0.0;
    }
  for (int i = 0; i < w; ++i)
    if (tid < cw) X[i * kU12Cols + tid] = A[(long long)(k0 + i) * lda + c0 + tid];
  __syncthreads();
  if (tid < cw) {
    double* x = X + tid;
    for (int t = 0; t < w; ++t) {
      const int p = piv[t];
      if (p != t) {
        const double v = x[t * kU12Cols];
        x[t * kU12Cols] = x[p * kU12Cols];
        x[p * kU12Cols] = v;
      }
    }
    if (right)
      for (int k = 0; k < w; ++k) {
        const double xk = x[k * kU12Cols];
        for (int i = k + 1; i < w; ++i) x[i * kU12Cols] = fma(-Ls[i * w + k], xk, x[i * kU12Cols]);
      }
  }
  __syncthreads();
  unsigned long long umax = 0ull;
  for (int i = 0; i < w; ++i)
    if (tid < cw) {
      const double v = X[i * kU12Cols + tid];
      A[(long long)(k0 + i) * lda + c0 + tid] = v;
      umax = max_bits(umax, abs_bits(v));
    }
  if (right) {
    for (int off = 16; off > 0; off >>= 1) umax = max_bits(umax, __shfl_xor_sync(0xffffffffu, umax, off));
    if (tid == 0) atomicMax(&st->umax_bits, umax);
  }
}

// Register-resident U12 for a full-width block (w == W): one thread per column, the
// column's W values in registers, GEPP's interchanges folded into the loads (each thread
// reads the block rows in their interchanged order), forward substitution with the unit
// lower L11 fully unrolled (L11 from shared memory, broadcast).  Left of the block only the
// interchanges apply.
template <int W>
__global__ void __launch_bounds__(32) u12_reg_kernel(double* __restrict__ A, long long lda, int n,
                                                     int k0, const int* __restrict__ ipiv,
                                                     int left_slices, int solve, DevState* st) {
  if (dev_status(st) != 0) return;
  __shared__ double Ls[W * W];
  __shared__ int src[W];
  const int tid = threadIdx.x;
  const bool side = blockIdx.x >= left_slices;      // right of the block
  const bool right = side && solve;                 // interchanges and the triangular solve
  const int c = side ? k0 + W + (blockIdx.x - left_slices) * 32 + tid : blockIdx.x * 32 + tid;
  const int cend = side ? n : k0;
  if (tid == 0) {                                  // composed row order of the interchanges
    for (int t = 0; t < W; ++t) src[t] = t;
    for (int t = 0; t < W; ++t) {
      const int p = ipiv[t];
      const int x = src[t]; src[t] = src[p]; src[p] = x;
    }
  }
  if (right)
    for (int e = tid; e < W * W; e += 32) {
      const int i = e / W, j = e - i * W;
      Ls[e] = (j < i) ? A[(long long)(k0 + i) * lda + k0 + j] : 0.0;
    }
  __syncthreads();
  const bool valid = c < cend;
  unsigned long long umax = 0ull;
  if (valid) {
    double x[W];
#pragma unroll
    for (int i = 0; i < W; ++i) x[i] = A[(long long)(k0 + src[i]) * lda + c];
    if (right) {
#pragma unroll
      for (int k = 0; k < W; ++k)
#pragma unroll
        for (int i = k + 1; i < W; ++i) x[i] = fma(-Ls[i * W + k], x[k], x[i]);
#pragma unroll
      for (int i = 0; i < W; ++i) umax = max_bits(umax, abs_bits(x[i]));
    }
#pragma unroll
    for (int i = 0; i < W; ++i) A[(long long)(k0 + i) * lda + c] = x[i];
  }
  if (right) {                                      // every lane takes part in the reduction
    for (int off = 16; off > 0; off >>= 1) umax = max_bits(umax, __shfl_xor_sync(0xffffffffu, umax, off));
    if (tid == 0) atomicMax(&st->umax_bits, umax);
  }
}

// Register-resident final multipliers for w == W: one thread per row below the block,
// row = (L21 with GEPP's column interchanges) * L11, fully unrolled.
template <int W>
__global__ void __launch_bounds__(32) lfix_reg_kernel(double* __restrict__ A, long long lda, int n,
                                                      int k0, const double* __restrict__ L21, int ldl21,
                                                      const int* __restrict__ ipiv, DevState* st) {
  if (dev_status(st) != 0) return;
  __shared__ double Ls[W * W];
  __shared__ int src[W];
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int t = 0; t < W; ++t) src[t] = t;
    for (int t = 0; t < W; ++t) {
      const int p = ipiv[t];
      const int x = src[t]; src[t] = src[p]; src[p] = x;
    }
  }
  for (int e = tid; e < W * W; e += 32) {
    const int i = e / W, j = e - i * W;
    Ls[e] = (j < i) ? A[(long long)(k0 + i) * lda + k0 + j] : 0.0;
  }
  __syncthreads();
  const int r = blockIdx.x * 32 + tid;             // row below the block
  if (r >= n - k0 - W) return;
  const double* l = L21 + (long long)r * ldl21;
  double x[W];
#pragma unroll
  for (int i = 0; i < W; ++i) x[i] = l[src[i]];
  double* out = A + (long long)(k0 + W + r) * lda + k0;
#pragma unroll
  for (int cc = 0; cc < W; ++cc) {
    double acc = x[cc];
#pragma unroll
    for (int i = cc + 1; i < W; ++i) acc = fma(x[i], Ls[i * W + cc], acc);
    out[cc] = acc;
  }
}

cudaError_t launch_u12(double* A, long long lda, int n, int k0, int w, const int* ipiv,
                       DevState* st, cudaStream_t s, int solve) {
  const int left = (k0 + kU12Cols - 1) / kU12Cols;
  const int right = (n - k0 - w + kU12Cols - 1) / kU12Cols;
  if (left + right == 0) return cudaSuccess;
  if (w == 64) {
    u12_reg_kernel<64><<<left + right, 32, 0, s>>>(A, lda, n, k0, ipiv, left, solve, st);
    return cudaGetLastError();
  }
  if (w == 16) {
    u12_reg_kernel<16><<<left + right, 32, 0, s>>>(A, lda, n, k0, ipiv, left, solve, st);
    return cudaGetLastError();
  }
  const size_t smem = (size_t)(w * w + w * kU12Cols) * sizeof(double);
  cudaError_t e = smem_optin(u12_kernel);
  if (e != cudaSuccess) return e;
  u12_kernel<<<left + right, kU12Cols, smem, s>>>(A, lda, n, k0, w, ipiv, left, solve, st);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- a7 on the tensor cores
//
// In the low-precision modes U12 = L11^-1 X (X: the block row after GEPP's interchanges)
// and the final multipliers (L21 Pi_jj) L11 run on the tensor-core update, written in its
// form C -= L U:  U12 = X - (I - L11^-1) X  and  (L21 Pi_jj) L11 = Y - Y (I - L11)  with
// Y = L21 Pi_jj.  This kernel forms E1 = I - L11^-1 and E2 = I - L11 (w x w each, ld w)
// from the unit lower L11 at A[k0][k0]; L11^-1 by forward substitution in FP32, one column
// per thread (the factors of these modes are FP32-accurate).
__global__ void __launch_bounds__(kMaxW) tri_blocks_kernel(const double* __restrict__ A, long long lda, int k0,
                                                           int w, double* __restrict__ E, DevState* st) {
  if (dev_status(st) != 0) return;
  extern __shared__ float shf[];
  float* Ls = shf;                         // strictly lower L11, w x w
  float* G = shf + w * w;                  // L11^-1, w x w
  const int t = threadIdx.x;
  for (int e = t; e < w * w; e += blockDim.x) {
    const int i = e / w, j = e - i * w;
    Ls[e] = j < i ? static_cast<float>(A[(long long)(k0 + i) * lda + k0 + j]) : 0.f;
  }
  __syncthreads();
  if (t < w) {
    for (int i = 0; i < w; ++i) {
      float acc = i == t ? 1.f : 0.f;
      for (int k = t; k < i; ++k) acc = fmaf(-Ls[i * w + k], G[k * w + t], acc);
      G[i * w + t] = acc;
    }
  }
  __syncthreads();
  for (int e = t; e < w * w; e += blockDim.x) {
    const int i = e / w, j = e - i * w;
    E[e] = (i == j ? 1.0 : 0.0) - static_cast<double>(G[e]);
    E[w * w + e] = j < i ? -A[(long long)(k0 + i) * lda + k0 + j] : 0.0;
  }
}

cudaError_t launch_tri_blocks(const double* A, long long lda, int k0, int w, double* E, DevState* st,
                              cudaStream_t s) {
  if (w <= 0 || w > kMaxW) return cudaErrorInvalidValue;
  cudaError_t e = smem_optin(tri_blocks_kernel);
  if (e != cudaSuccess) return e;
  tri_blocks_kernel<<<1, kMaxW, 2 * (size_t)w * w * sizeof(float), s>>>(A, lda, k0, w, E, st);
  return cudaGetLastError();
}

// A[k0 + w + r][k0 + c] = L21[r][src(c)]: the multipliers with GEPP's column interchanges,
// the operand Y above.
__global__ void lfix_copy_kernel(double* __restrict__ A, long long lda, int rows, int k0, int w,
                                 const double* __restrict__ L21, int ldl21, const int* __restrict__ ipiv,
                                 DevState* st) {
  if (dev_status(st) != 0) return;
  __shared__ int src[kMaxW];
  if (threadIdx.x == 0) {
    for (int t = 0; t < w; ++t) src[t] = t;
    for (int t = 0; t < w; ++t) {
      const int p = ipiv[t];
      const int x = src[t]; src[t] = src[p]; src[p] = x;
    }
  }
  __syncthreads();
  const long long total = (long long)rows * w;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / w), c = (int)(e - (long long)r * w);
    A[(long long)(k0 + w + r) * lda + k0 + c] = L21[(long long)r * ldl21 + src[c]];
  }
}

cudaError_t launch_lfix_copy(double* A, long long lda, int n, int k0, int w, const double* L21, int ldl21,
                             const int* ipiv, DevState* st, cudaStream_t s) {
  const int rows = n - k0 - w;
  if (rows <= 0) return cudaSuccess;
  const long long total = (long long)rows * w;
  lfix_copy_kernel<<<(int)std::min<long long>((total + 255) / 256, 152 * 8), 256, 0, s>>>(A, lda, rows, k0, w, L21,
                                                                                        ldl21, ipiv, st);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- final L below the block
constexpr int kLfixRows = 32;

__global__ void __launch_bounds__(kLfixRows) lfix_kernel(double* __restrict__ A, long long lda, int n,
                                                         int k0, int w, const double* __restrict__ L21,
                                                         int ldl21, const int* __restrict__ ipiv,
                                                         DevState* st) {
  if (dev_status(st) != 0) return;
  extern __shared__ double sh[];
  double* Ls = sh;                       // w x w unit lower L11
  double* X = sh + w * w;                // kLfixRows x (w + 1)
  __shared__ int piv[kMaxW];
  const int WP = w + 1;
  const int tid = threadIdx.x;
  const int rbase = blockIdx.x * kLfixRows;
  const int rows = min(kLfixRows, n - k0 - w - rbase);
  for (int t = tid; t < w; t += blockDim.x) piv[t] = ipiv[t];
  for (int e = tid; e < w * w; e += blockDim.x) {
    const int i = e / w, j = e - i * w;
    Ls[e] = (j < i) ? A[(long long)(k0 + i) * lda + k0 + j] : (i == j ? 1.0 : 0.0);
  }
  for (int e = tid; e < rows * w; e += blockDim.x) {
    const int r = e / w, j = e - r * w;
    X[r * WP + j] = L21[(long long)(rbase + r) * ldl21 + j];
  }
  __syncthreads();
  if (tid < rows) {
    double* x = X + tid * WP;
    for (int t = 0; t < w; ++t) {
      const int p = piv[t];
      if (p != t) { const double v = x[t]; x[t] = x[p]; x[p] = v; }
    }
    // x <- x * L11, in place from the left column: out_c = x_c + sum_{i > c} x_i L11(i, c)
    for (int c = 0; c < w; ++c) {
      double acc = x[c];
      for (int i = c + 1; i < w; ++i) acc = fma(x[i], Ls[i * w + c], acc);
      x[c] = acc;
    }
  }
  __syncthreads();
  for (int e = tid; e < rows * w; e += blockDim.x) {
    const int r = e / w, j = e - r * w;
    A[(long long)(k0 + w + rbase + r) * lda + k0 + j] = X[r * WP + j];
  }
}

cudaError_t launch_lfix(double* A, long long lda, int n, int k0, int w, const double* L21,
                        int ldl21, const int* ipiv, DevState* st, cudaStream_t s) {
  const int rows = n - k0 - w;
  if (rows <= 0) return cudaSuccess;
  if (w == 64) {
    lfix_reg_kernel<64><<<(rows + 31) / 32, 32, 0, s>>>(A, lda, n, k0, L21, ldl21, ipiv, st);
    return cudaGetLastError();
  }
  if (w == 16) {
    lfix_reg_kernel<16><<<(rows + 31) / 32, 32, 0, s>>>(A, lda, n, k0, L21, ldl21, ipiv, st);
    return cudaGetLastError();
  }
  const size_t smem = (size_t)(w * w + kLfixRows * (w + 1)) * sizeof(double);
  cudaError_t e = smem_optin(lfix_kernel);
  if (e != cudaSuccess) return e;
  lfix_kernel<<<(rows + kLfixRows - 1) / kLfixRows, kLfixRows, smem, s>>>(A, lda, n, k0, w, L21,
                                                                          ldl21, ipiv, st);
  return cudaGetLastError();
}

}  // namespace prrp

namespace prrp {

// Self-test of the bounded wait: CTA 0 waits at a grid barrier that CTA 1 never reaches,
// so the wait must run out after st->spin_limit polls and record PRRP_ERR_TIMEOUT.
__global__ void wait_selftest_kernel(DevState* st) {
  if (blockIdx.x == 1) return;            // never arrives
  grid_barrier(st, gridDim.x, 99);
}

cudaError_t launch_wait_selftest(DevState* st, cudaStream_t s) {
  void* args[] = {&st};
  return cudaLaunchCooperativeKernel((const void*)wait_selftest_kernel, dim3(2), dim3(32), args, 0, s);
}

}  // namespace prrp
