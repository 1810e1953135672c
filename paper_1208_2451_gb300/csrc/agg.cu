// Aggregated trailing update of the mixed-precision forms: the Schur update of Algorithm 1
// (line 7) applied to the columns right of a block of NB = q b columns once per block, as
// one rank-NB tensor-core product, instead of once per panel as q rank-b products.
//
// Inside the block the panels run as in Algorithm 1, but their row interchanges, Schur
// updates and U12 touch only the block's own columns (and the columns of L on the left).
// At the block's end, with F the columns right of the block, K0..KB the block's rows,
// P_blk the block's composed row order, L_blk the NB x NB unit lower triangle of the
// block's final multipliers and L2 the final multipliers of the rows below the block:
//     A(K0:n, F)  <- P_blk A(K0:n, F)             (only the rows the block moved)
//     U(K0:KB, F)  = L_blk^-1 A(K0:KB, F)         (panel by panel, tensor cores)
//     A(KB:n, F) -= L2 U(K0:KB, F)                (one rank-NB update, tensor cores)
// This is the per-panel sequence up to rounding: a panel's update L21 A12 equals
// (L21 Pi_jj^T L11)(L11^-1 Pi_jj A12), its final multipliers times its U12 rows, and the
// U12 rows of the block's panels, taken together, solve L_blk U = A(K0:KB, F).  The solve
// goes panel by panel (the rows of panel t lose the earlier panels' final multipliers
// times their U rows, then take L11^-1 as the per-panel U12 does), not through an explicit
// L_blk^-1: with the block's final multipliers off the diagonal blocks, that inverse grows
// with the block and its product on the tensor cores lost accuracy on ill-conditioned A.
//
// This file holds the helpers of the block's end: the moved rows (from the row order at
// the block's start and at its end) and the moves over a column range.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace prrp {

// pos0[perm0[q]] = q: where each row of the block's start sat.
__global__ void block_pos_kernel(const int* __restrict__ perm0, int rows, int* __restrict__ pos0) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < rows; q += gridDim.x * blockDim.x) pos0[perm0[q]] = q;
}

// Every position i whose row came from another position: (i, src) appended to pairs.
__global__ void block_pairs_kernel(const int* __restrict__ perm, int K0, int rows, const int* __restrict__ pos0,
                                   int* __restrict__ pairs, int* __restrict__ count, int cap, DevState* st) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) {
    const int src = pos0[perm[K0 + i]];
    if (src != i) {
      const int q = atomicAdd(count, 1);
      if (q < cap) {
        pairs[2 * q] = i;
        pairs[2 * q + 1] = src;
      } else {
        set_error(st, PRRP_ERR_UNSUPPORTED);    // not reached: cap bounds the rows a block moves
      }
    }
  }
}

cudaError_t launch_block_pairs(const int* perm0, const int* perm, int K0, int rows, int* pos0, int* pairs,
                               int* count, int cap, DevState* st, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const int grid = std::min((rows + 255) / 256, 152 * 4);
  block_pos_kernel<<<grid, 256, 0, s>>>(perm0, rows, pos0);
  block_pairs_kernel<<<grid, 256, 0, s>>>(perm, K0, rows, pos0, pairs, count, cap, st);
  return cudaGetLastError();
}

// tmp[q][c] = A[K0 + src_q][c0 + c], then A[K0 + dst_q][c0 + c] = tmp[q][c].
__global__ void block_gather_kernel(const double* __restrict__ A, long long lda, int K0, int c0, int nc,
                                    const int* __restrict__ pairs, const int* __restrict__ count, int cap,
                                    double* __restrict__ tmp, DevState* st) {
  if (dev_status(st) != 0) return;
  const long long total = (long long)min(*count, cap) * nc;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(e / nc), c = (int)(e - (long long)q * nc);
    tmp[e] = A[(long long)(K0 + pairs[2 * q + 1]) * lda + c0 + c];
  }
}

__global__ void block_scatter_kernel(double* __restrict__ A, long long lda, int K0, int c0, int nc,
                                     const int* __restrict__ pairs, const int* __restrict__ count, int cap,
                                     const double* __restrict__ tmp, DevState* st) {
  if (dev_status(st) != 0) return;
  const long long total = (long long)min(*count, cap) * nc;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(e / nc), c = (int)(e - (long long)q * nc);
    A[(long long)(K0 + pairs[2 * q]) * lda + c0 + c] = tmp[e];
  }
}

cudaError_t launch_block_moves(double* A, long long lda, int K0, int c0, int nc, const int* pairs,
                               const int* count, int cap, double* tmp, DevState* st, cudaStream_t s) {
  if (nc <= 0 || cap <= 0) return cudaSuccess;
  const long long most = (long long)cap * nc;
  const int grid = (int)std::min<long long>((most + 255) / 256, 152 * 8);
  block_gather_kernel<<<grid, 256, 0, s>>>(A, lda, K0, c0, nc, pairs, count, cap, tmp, st);
  block_scatter_kernel<<<grid, 256, 0, s>>>(A, lda, K0, c0, nc, pairs, count, cap, tmp, st);
  return cudaGetLastError();
}

}  // namespace prrp
