// Triangular solves and FP64 residuals with the in-place L\U of LU_PRRP (the solver tests
// of Section 2.3; the refinement of Section 3.3).
//
// Forward and back substitution are blocked by 64 rows.  Launch j updates every later row
// block with the 64 unknowns of block j (a GEMV/GEMM strip, HBM-bound on L or U), and the
// CTA that owns block j+1 then solves its 64 x 64 triangle with one warp per right-hand
// side (shuffle broadcast of each solved unknown), so the next launch can use it.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace prrp {

constexpr int kSB = 64;          // solve block rows
constexpr int kSolveThreads = 256;

__global__ void gather_rows_kernel(const double* __restrict__ B, long long ldb,
                                   const int* __restrict__ perm, int n, int nrhs,
                                   double* __restrict__ Y) {
  const long long total = (long long)n * nrhs;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / nrhs), c = (int)(e - (long long)i * nrhs);
    Y[e] = B[(long long)perm[i] * ldb + c];
  }
}

cudaError_t launch_gather_rows(const double* B, long long ldb, const int* perm, int n, int nrhs,
                               double* Y, cudaStream_t s) {
  const long long total = (long long)n * nrhs;
  if (total == 0) return cudaSuccess;
  const int grid = (int)std::min<long long>((total + 255) / 256, 152 * 16);
  gather_rows_kernel<<<grid, 256, 0, s>>>(B, ldb, perm, n, nrhs, Y);
  return cudaGetLastError();
}

// Solve the kb x kb triangle at rows [r0, r0 + kb) of Y in place, one warp per column.
// lower: unit lower L; otherwise upper U (divides by the diagonal).
__device__ void solve_diag_block(const double* __restrict__ LU, long long lda, double* Y,
                                 int nrhs, int r0, int kb, bool lower) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  for (int c = warp; c < nrhs; c += nwarps) {
    // lane holds rows r0 + lane and r0 + lane + 32
    double y0 = lane < kb ? Y[(long long)(r0 + lane) * nrhs + c] : 0.0;
    double y1 = lane + 32 < kb ? Y[(long long)(r0 + lane + 32) * nrhs + c] : 0.0;
    if (lower) {
      for (int k = 0; k < kb; ++k) {
        const double xk = __shfl_sync(0xffffffffu, k < 32 ? y0 : y1, k & 31);
        const int i0 = lane, i1 = lane + 32;
        if (i0 > k && i0 < kb) y0 = fma(-LU[(long long)(r0 + i0) * lda + r0 + k], xk, y0);
        if (i1 > k && i1 < kb) y1 = fma(-LU[(long long)(r0 + i1) * lda + r0 + k], xk, y1);
      }
    } else {
      for (int k = kb - 1; k >= 0; --k) {
        const int ko = k & 31;
        if (k < 32) { if (lane == ko) y0 = y0 / LU[(long long)(r0 + k) * lda + r0 + k]; }
        else        { if (lane == ko) y1 = y1 / LU[(long long)(r0 + k) * lda + r0 + k]; }
        const double xk = __shfl_sync(0xffffffffu, k < 32 ? y0 : y1, ko);
        const int i0 = lane, i1 = lane + 32;
        if (i0 < k) y0 = fma(-LU[(long long)(r0 + i0) * lda + r0 + k], xk, y0);
        if (i1 < k) y1 = fma(-LU[(long long)(r0 + i1) * lda + r0 + k], xk, y1);
      }
    }
    if (lane < kb) Y[(long long)(r0 + lane) * nrhs + c] = y0;
    if (lane + 32 < kb) Y[(long long)(r0 + lane + 32) * nrhs + c] = y1;
  }
}

// One step of blocked substitution.  jb = block just solved (-1: none yet).  CTA b updates
// row block `blk` with the solved unknowns of jb: one warp per row, lanes along k (each
// row of the 64 x 64 block is two coalesced 256-byte loads), the 64 solved unknowns of
// each right-hand side staged in shared memory.  The CTA of the block that becomes final
// next then solves its triangle.
constexpr int kStageRhs = 32;    // right-hand sides staged per pass

__global__ void __launch_bounds__(kSolveThreads) trsv_step_kernel(const double* __restrict__ LU,
                                                                  long long lda, int n, double* Y,
                                                                  int nrhs, int jb, int lower) {
  __shared__ double xs[kSB * kStageRhs];
  const int nb = (n + kSB - 1) / kSB;
  int blk, next;
  if (lower) { blk = jb + 1 + blockIdx.x; next = jb + 1; }
  else       { blk = (jb < 0 ? nb : jb) - 1 - blockIdx.x; next = (jb < 0 ? nb : jb) - 1; }
  if (blk < 0 || blk >= nb) return;
  const int r0 = blk * kSB, kb = min(kSB, n - r0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  if (jb >= 0) {
    const int c0 = jb * kSB, kc = min(kSB, n - c0);
    for (int cb = 0; cb < nrhs; cb += kStageRhs) {
      const int nc = min(kStageRhs, nrhs - cb);
      __syncthreads();
      for (int e = threadIdx.x; e < kc * nc; e += blockDim.x) {
        const int k = e / nc, c = e - k * nc;
        xs[k * kStageRhs + c] = Y[(long long)(c0 + k) * nrhs + cb + c];
      }
      __syncthreads();
      // Y[r0:r0+kb, cb:cb+nc] -= LU[r0:r0+kb, c0:c0+kc] * xs
      for (int i = warp; i < kb; i += nwarps) {
        const double* a = LU + (long long)(r0 + i) * lda + c0;
        const double a0 = lane < kc ? a[lane] : 0.0;
        const double a1 = lane + 32 < kc ? a[lane + 32] : 0.0;
        for (int c = 0; c < nc; ++c) {
          double acc = a0 * (lane < kc ? xs[lane * kStageRhs + c] : 0.0);
          if (lane + 32 < kc) acc = fma(a1, xs[(lane + 32) * kStageRhs + c], acc);
          for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
          if (lane == 0) Y[(long long)(r0 + i) * nrhs + cb + c] -= acc;
        }
      }
    }
    __syncthreads();
  }
  if (blk == next) solve_diag_block(LU, lda, Y, nrhs, r0, kb, lower != 0);
}

static cudaError_t trsv(const double* LU, long long lda, int n, double* Y, int nrhs, bool lower,
                        cudaStream_t s) {
  if (n == 0 || nrhs == 0) return cudaSuccess;
  const int nb = (n + kSB - 1) / kSB;
  // first launch: solve the first block only; then nb - 1 update+solve launches, the last
  // update launch needs no further solve.
  trsv_step_kernel<<<1, kSolveThreads, 0, s>>>(LU, lda, n, Y, nrhs, -1, lower);
  for (int j = 0; j < nb - 1; ++j) {
    const int jb = lower ? j : nb - 1 - j;
    trsv_step_kernel<<<nb - 1 - j, kSolveThreads, 0, s>>>(LU, lda, n, Y, nrhs, jb, lower);
  }
  return cudaGetLastError();
}

cudaError_t launch_trsv_lower_unit(const double* LU, long long lda, int n, double* Y, int nrhs,
                                   cudaStream_t s) {
  return trsv(LU, lda, n, Y, nrhs, true, s);
}

cudaError_t launch_trsv_upper(const double* LU, long long lda, int n, double* Y, int nrhs,
                              cudaStream_t s) {
  return trsv(LU, lda, n, Y, nrhs, false, s);
}

// R = B - A X (FP64), one CTA per row (coalesced row reads).  The 1-norm numerators of
// eta are reduced afterwards by residual_norms_kernel in a fixed order, so the refinement's
// stopping decisions, and with them the returned bits, do not depend on scheduling.
__global__ void __launch_bounds__(kSolveThreads) residual_kernel(const double* __restrict__ A,
                                                                 long long lda, int n,
                                                                 const double* __restrict__ X,
                                                                 long long ldx,
                                                                 int nrhs, const double* __restrict__ B,
                                                                 long long ldb, double* __restrict__ R) {
  __shared__ double part[kSolveThreads / 32];
  for (int row = blockIdx.x; row < n; row += gridDim.x) {
    const double* a = A + (long long)row * lda;
    for (int c = 0; c < nrhs; ++c) {
      double acc = 0.0;
      for (int k = threadIdx.x; k < n; k += blockDim.x) acc = fma(a[k], X[(long long)k * ldx + c], acc);
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
      __syncthreads();
      if (threadIdx.x == 0) {
        double ax = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) ax += part[q];
        R[(long long)row * nrhs + c] = B[(long long)row * ldb + c] - ax;
      }
      __syncthreads();
    }
  }
}

// norms[c] = ||R(:,c)||_1, norms[nrhs + c] = ||X(:,c)||_1, norms[2 nrhs + c] = ||B(:,c)||_1;
// one CTA per column, each thread a fixed stride of rows, then a fixed-order tree.
__global__ void __launch_bounds__(kSolveThreads) residual_norms_kernel(const double* __restrict__ R, int n,
                                                                       const double* __restrict__ X, long long ldx,
                                                                       int nrhs, const double* __restrict__ B,
                                                                       long long ldb, double* norms) {
  __shared__ double sr[kSolveThreads], sx[kSolveThreads], sb[kSolveThreads];
  const int c = blockIdx.x;
  double r = 0.0, x = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    r += abs_int(R[(long long)i * nrhs + c]);
    x += abs_int(X[(long long)i * ldx + c]);
    b += abs_int(B[(long long)i * ldb + c]);
  }
  sr[threadIdx.x] = r; sx[threadIdx.x] = x; sb[threadIdx.x] = b;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      sr[threadIdx.x] += sr[threadIdx.x + h];
      sx[threadIdx.x] += sx[threadIdx.x + h];
      sb[threadIdx.x] += sb[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { norms[c] = sr[0]; norms[nrhs + c] = sx[0]; norms[2 * nrhs + c] = sb[0]; }
}

cudaError_t launch_residual(const double* A, long long lda, int n, const double* X, long long ldx,
                            int nrhs, const double* B, long long ldb, double* R, double* norms,
                            cudaStream_t s) {
  if (n == 0 || nrhs == 0) return cudaSuccess;
  residual_kernel<<<std::min(n, 152 * 8), kSolveThreads, 0, s>>>(A, lda, n, X, ldx, nrhs, B, ldb, R);
  residual_norms_kernel<<<nrhs, kSolveThreads, 0, s>>>(R, n, X, ldx, nrhs, B, ldb, norms);
  return cudaGetLastError();
}

// out = max_j sum_i |a_ij| (the matrix 1-norm), one thread per column.
__global__ void norm1_kernel(const double* __restrict__ A, long long lda, int n, double* out) {
  double best = 0.0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += abs_int(A[(long long)i * lda + j]);
    best = fmax(best, s);
  }
  for (int off = 16; off > 0; off >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, off));
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(reinterpret_cast<unsigned long long*>(out), best);
}

cudaError_t launch_norm1(const double* A, long long lda, int n, double* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), s);
  if (e != cudaSuccess || n == 0) return e;
  norm1_kernel<<<std::max(1, std::min((n + 127) / 128, 152 * 4)), 128, 0, s>>>(A, lda, n, out);
  return cudaGetLastError();
}

__global__ void axpy_rows_kernel(double* X, long long ldx, const double* D, double alpha, int n,
                                 int nrhs) {
  const long long total = (long long)n * nrhs;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / nrhs), c = (int)(e - (long long)i * nrhs);
    X[(long long)i * ldx + c] = fma(alpha, D[e], X[(long long)i * ldx + c]);
  }
}

cudaError_t launch_axpy_rows(double* X, long long ldx, const double* D, double alpha, int n,
                             int nrhs, cudaStream_t s) {
  const long long total = (long long)n * nrhs;
  if (total == 0) return cudaSuccess;
  axpy_rows_kernel<<<(int)std::min<long long>((total + 255) / 256, 152 * 16), 256, 0, s>>>(X, ldx, D, alpha, n, nrhs);
  return cudaGetLastError();
}

__global__ void copy_rows_kernel(const double* src, long long lds, double* dst, long long ldd,
                                 int n, int ncols) {
  const long long total = (long long)n * ncols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / ncols), c = (int)(e - (long long)i * ncols);
    dst[(long long)i * ldd + c] = src[(long long)i * lds + c];
  }
}

cudaError_t launch_copy_rows(const double* src, long long lds, double* dst, long long ldd, int n,
                             int ncols, cudaStream_t s) {
  const long long total = (long long)n * ncols;
  if (total == 0) return cudaSuccess;
  copy_rows_kernel<<<(int)std::min<long long>((total + 255) / 256, 152 * 16), 256, 0, s>>>(src, lds, dst, ldd, n, ncols);
  return cudaGetLastError();
}

}  // namespace prrp
