// Triangular solves and FP64 residuals with the in-place L\U of LU_PRRP (the solver tests
// of Section 2.3; the refinement of Section 3.3).
//
// Forward and back substitution are blocked by 64 rows with inverted diagonal blocks: one
// launch per triangle for up to 16 right-hand sides (CTAs following an in-order front of
// final blocks), else one launch per block.  The refinement residual is always FP64;
// factors from a low-precision Schur update are applied in FP32 for the correction solves,
// and the block products and column operations below serve the GMRES-based refinement.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace prrp {

constexpr int kSB = 64;          // solve block rows
constexpr int kSolveThreads = 256;
constexpr int kB1 = kSB + 1;   // padded row of a staged diagonal block

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

// ---------------------------------------------------------------- blocked substitution
//
// Diagonal blocks are inverted once per factorization (invert_diag_kernel), so solving a
// 64 x 64 triangle is a small GEMV instead of a 64-step dependent chain.  Substitution
// step j then is one launch: every CTA owns a 16-row chunk of a later row block and
// subtracts L_ij x_j (forward) or U_ij x_j (backward) from it; the CTA that completes the
// last chunk of the next block (a counter per block, fenced) applies that block's inverse,
// making x_{j+1} (x_{j-1}) final for the next launch.  T = double or float.

constexpr int kRC = 16;          // rows per chunk CTA
constexpr int kXS = 16;          // right-hand sides staged per pass
constexpr int kXP = kXS + 1;     // padded row of the staged unknowns (conflict-free split-k reads)

// Column t of the inverse of one diagonal block, by substitution against e_t, all columns
// in lockstep (thread t).  blockIdx.y = 0: unit lower L; 1: upper U.
template <typename T>
__global__ void __launch_bounds__(kSB) invert_diag_kernel(const double* __restrict__ LU, long long lda, int n,
                                                         T* __restrict__ Dinv) {
  extern __shared__ double dsm[];
  double* S = dsm;                    // the block, rows padded to kB1
  double* X = S + kSB * kB1;          // the inverse, column t owned by thread t
  double* rd = X + kSB * kB1;         // reciprocals of the diagonal
  const int nb = (n + kSB - 1) / kSB, b = blockIdx.x, upper = blockIdx.y;
  const int r0 = b * kSB, kb = min(kSB, n - r0), t = threadIdx.x;
  for (int e = t; e < kSB * kSB; e += kSB) {
    const int i = e / kSB, k = e - i * kSB;
    S[i * (kSB + 1) + k] = (i < kb && k < kb) ? LU[(long long)(r0 + i) * lda + r0 + k] : 0.0;
  }
  __syncthreads();
  rd[t] = t < kb ? 1.0 / S[t * kB1 + t] : 0.0;
  __syncthreads();
  if (!upper) {
    for (int i = 0; i < kb; ++i) {
      double acc = 0.0;
      for (int k = 0; k < i; ++k) acc = fma(S[i * kB1 + k], X[k * kB1 + t], acc);
      X[i * kB1 + t] = (i == t) ? 1.0 : (i > t ? -acc : 0.0);
    }
  } else {
    for (int i = kb - 1; i >= 0; --i) {
      double acc = 0.0;
      for (int k = i + 1; k < kb; ++k) acc = fma(S[i * kB1 + k], X[k * kB1 + t], acc);
      X[i * kB1 + t] = (i == t) ? rd[i] : (i < t ? -acc * rd[i] : 0.0);
    }
  }
  __syncthreads();
  T* out = Dinv + ((size_t)upper * nb + b) * kSB * kSB;
  for (int e = t; e < kSB * kSB; e += kSB) {
    const int i = e / kSB, k = e - i * kSB;
    out[e] = static_cast<T>((i < kb && k < kb) ? X[i * kB1 + k] : 0.0);
  }
}

// Y[rows] -= M[rows, c0:c0+kc] * Xs for `nr` rows of one chunk.  Ms: nr x kSB, Xs: kSB x kXP
// in shared memory; the outputs (row, column) are split over the CTA with `sk` threads per
// output summing interleaved k and reducing by shuffles (fixed order: deterministic).
template <typename T>
__device__ __forceinline__ void chunk_gemv(const T* Ms, const T* Xs, int nr, int kc, int nc, T* Y, int ldy,
                                           int row0, int col0, bool subtract) {
  const int outs = nr * nc;
  int sk = 1;
  while (sk < 16 && outs * sk * 2 <= kSolveThreads) sk *= 2;
  const int kk = threadIdx.x & (sk - 1);
  for (int o = threadIdx.x / sk; o < ((outs + (kSolveThreads / sk) - 1) / (kSolveThreads / sk)) * (kSolveThreads / sk);
       o += kSolveThreads / sk) {
    const bool live = o < outs;
    const int i = live ? o / nc : 0, c = live ? o - (o / nc) * nc : 0;
    T acc0 = 0, acc1 = 0;
    if (live) {
      int k = kk;
      for (; k + sk < kc; k += 2 * sk) {
        acc0 = fma(Ms[i * kSB + k], Xs[k * kXP + c], acc0);
        acc1 = fma(Ms[i * kSB + k + sk], Xs[(k + sk) * kXP + c], acc1);
      }
      if (k < kc) acc0 = fma(Ms[i * kSB + k], Xs[k * kXP + c], acc0);
    }
    T acc = acc0 + acc1;
    for (int off = 1; off < sk; off <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (live && kk == 0) {
      T* y = Y + (long long)(row0 + i) * ldy + col0 + c;
      *y = subtract ? *y - acc : acc;
    }
  }
}

// x_b = Dinv_b y_b for block b (rows r0 .. r0 + kb), all right-hand sides, in place.
template <typename T>
__device__ void apply_inverse(const T* __restrict__ D, T* Y, int nrhs, int r0, int kb, T* Ms, T* Xs) {
  for (int e = threadIdx.x; e < kSB * kSB; e += blockDim.x) Ms[e] = D[e];
  for (int cb = 0; cb < nrhs; cb += kXS) {
    const int nc = min(kXS, nrhs - cb);
    __syncthreads();
    for (int e = threadIdx.x; e < kSB * nc; e += blockDim.x) {
      const int k = e / nc, c = e - k * nc;
      Xs[k * kXP + c] = k < kb ? __ldcg(&Y[(long long)(r0 + k) * nrhs + cb + c]) : T(0);
    }
    __syncthreads();
    chunk_gemv(Ms, Xs, kb, kb, nc, Y, nrhs, r0, cb, false);
  }
}

template <typename T>
__global__ void __launch_bounds__(kSolveThreads) trsv_first_kernel(const T* __restrict__ Dinv, int n, T* Y,
                                                                   int nrhs, int lower) {
  __shared__ T Ms[kSB * kSB];
  __shared__ T Xs[kSB * kXP];
  const int nb = (n + kSB - 1) / kSB, b = lower ? 0 : nb - 1;
  const int r0 = b * kSB, kb = min(kSB, n - r0);
  apply_inverse(Dinv + ((size_t)(lower ? 0 : 1) * nb + b) * kSB * kSB, Y, nrhs, r0, kb, Ms, Xs);
}

template <typename T>
__global__ void __launch_bounds__(kSolveThreads) trsv_step_kernel(const T* __restrict__ LU, long long lda,
                                                                  const T* __restrict__ Dinv, int n, T* Y,
                                                                  int nrhs, int j, int lower,
                                                                  unsigned* __restrict__ counters) {
  __shared__ T Ms[kSB * kSB];      // the chunk's rows of L or U, later the next block's inverse
  __shared__ T Xs[kSB * kXP];
  __shared__ int s_last;
  const int nb = (n + kSB - 1) / kSB;
  const int per = kSB / kRC;                       // chunks per block
  const int blk = lower ? j + 1 + (int)blockIdx.x / per : j - 1 - (int)blockIdx.x / per;
  const int next = lower ? j + 1 : j - 1;
  const int r0 = blk * kSB + ((int)blockIdx.x % per) * kRC;
  const int nr = max(0, min(kRC, n - r0));
  const int c0 = j * kSB, kc = min(kSB, n - c0);
  for (int e = threadIdx.x; e < kRC * kSB; e += blockDim.x) {
    const int i = e / kSB, k = e - i * kSB;
    Ms[e] = (i < nr && k < kc) ? LU[(long long)(r0 + i) * lda + c0 + k] : T(0);
  }
  for (int cb = 0; cb < nrhs; cb += kXS) {
    const int nc = min(kXS, nrhs - cb);
    __syncthreads();
    for (int e = threadIdx.x; e < kSB * nc; e += blockDim.x) {
      const int k = e / nc, c = e - k * nc;
      Xs[k * kXP + c] = k < kc ? Y[(long long)(c0 + k) * nrhs + cb + c] : T(0);
    }
    __syncthreads();
    if (nr > 0) chunk_gemv(Ms, Xs, nr, kc, nc, Y, nrhs, r0, cb, true);
  }
  if (blk != next) return;
  // the last chunk of the next block to finish makes its unknowns final
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    // every chunk CTA of the block counts, also those past the matrix edge (no rows)
    s_last = atomicAdd(&counters[next], 1u) == (unsigned)(per - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int nr0 = next * kSB;
  apply_inverse(Dinv + ((size_t)(lower ? 0 : 1) * nb + next) * kSB * kSB, Y, nrhs, nr0, min(kSB, n - nr0), Ms, Xs);
}

template <typename T>
static cudaError_t trsv_t(const T* LU, long long lda, const T* Dinv, int n, T* Y, int nrhs, bool lower,
                          unsigned* counters, cudaStream_t s) {
  if (n == 0 || nrhs == 0) return cudaSuccess;
  const int nb = (n + kSB - 1) / kSB, per = kSB / kRC;
  cudaError_t e = cudaMemsetAsync(counters, 0, sizeof(unsigned) * nb, s);
  if (e != cudaSuccess) return e;
  trsv_first_kernel<T><<<1, kSolveThreads, 0, s>>>(Dinv, n, Y, nrhs, lower);
  for (int q = 0; q < nb - 1; ++q) {
    const int j = lower ? q : nb - 1 - q;
    trsv_step_kernel<T><<<(nb - 1 - q) * per, kSolveThreads, 0, s>>>(LU, lda, Dinv, n, Y, nrhs, j, lower,
                                                                       counters);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- one-launch substitution
//
// For up to kXS right-hand sides a whole triangle is solved by one launch instead of one
// launch per row block.  CTAs take tickets in the order they start; ticket t owns chunk
// t % per (RC rows) of row block t / per in solve order (top down for L, bottom up for U).
// A chunk streams its rows' off-diagonal tiles M_bj and subtracts M_bj x_j as soon as
// block j is final (a "front" counter: the number of blocks final so far, in order, so one
// poll can clear many tiles), then the block's chunks share their part of y_b and each
// computes its rows of x_b = Dinv_b y_b.  A CTA waits only on smaller tickets or on the
// other chunks of its own block, and those started before any CTA of a later block took
// its ticket, so the chain needs no co-residency guarantee beyond one block's chunks.
//
// Waiting is graded by urgency: a CTA whose own block is more than two blocks past the
// front backs off in proportion to that distance, so that the few CTAs next in line are
// the ones polling the front's cache line.  Every wait is bounded (DevState::spin_limit,
// else kSpinLimit, in units of 32 ns of back-off); a wait that runs out records its site
// in counter word 0 and every CTA returns at its next wait.
//
// Counter words: [0] site of a wait that ran out (0: none; cleared by the host), [1] ticket,
// [kFrontWord] front (a cache line of its own), [kReadyWord + p] chunks of block p that
// published y, [kReadyWord + nb + p] chunks that wrote x.

constexpr int kFrontWord = 32;
constexpr int kReadyWord = 64;
static_assert(kReadyWord == kTrsvCounterHead, "counter layout");

__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned atom_acq_rel_add(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Polls *flag until it reaches target.  own >= 0: the caller's own block in solve order,
// which grades the back-off by its distance from the observed value; own < 0: poll fast.
// Returns false when the wait runs out or another CTA's did.
__device__ __forceinline__ bool chain_wait(const unsigned* flag, unsigned target, int own, unsigned* err,
                                           unsigned limit, unsigned site, unsigned* seen) {
  unsigned v, spent = 0;
  while ((v = ld_acquire_u32(flag)) < target) {
    if (*((volatile unsigned*)err) != 0) return false;
    const int gap = own - (int)v;
    const unsigned ns = (own >= 0 && gap > 2) ? min(256u * (unsigned)gap, 4096u) : 32u;
    spent += ns >> 5;
    if (spent > limit) {
      atomicCAS(err, 0u, site);
      return false;
    }
    __nanosleep(ns);
  }
  *seen = v;
  return true;
}

// Sum over the KT consecutive lanes that share one row (butterfly: fixed order).
template <int KT, int NC, typename T>
__device__ __forceinline__ void row_sum(T (&v)[NC], int nrhs) {
#pragma unroll
  for (int cc = 0; cc < NC; ++cc) {
    if (cc < nrhs) {
#pragma unroll
      for (int off = 1; off < KT; off <<= 1) v[cc] += __shfl_xor_sync(0xffffffffu, v[cc], off);
    }
  }
}

template <typename T, int RC, int NC>
__global__ void __launch_bounds__(kSolveThreads) trsv_chain_kernel(const T* __restrict__ LU, long long lda,
                                                                   const T* __restrict__ Dinv, int n, T* In,
                                                                   T* Out, int nrhs, int lower, unsigned* c,
                                                                   const DevState* __restrict__ st) {
  constexpr int KT = kSolveThreads / RC;   // threads per row, consecutive lanes
  constexpr int KS = kSB / KT;             // columns per thread, interleaved by KT
  constexpr int per = kSB / RC;            // chunk CTAs per row block
  static_assert(KT <= 32 && KT * RC == kSolveThreads && KS * KT == kSB && NC <= kXS, "chunk shape");
  __shared__ T xs[kSB * kXP];
  __shared__ unsigned s_t, s_front;
  __shared__ int s_ok;
  const int nb = (n + kSB - 1) / kSB;
  unsigned* err = c;
  unsigned* front = c + kFrontWord;
  unsigned* ready = c + kReadyWord;
  unsigned* done = ready + nb;
  const int tid = threadIdx.x;
  if (tid == 0) {
    s_t = atomicAdd(c + 1, 1u);
    s_front = 0;
  }
  __syncthreads();
  const int t = (int)s_t;
  const int p = t / per, ch = t - p * per;
  const int b = lower ? p : nb - 1 - p;
  const int r = tid / KT, q = tid - r * KT;
  const int rb = ch * RC + r;              // row within the block
  const int row = b * kSB + rb;
  const bool live = row < n;
  const unsigned limit = st->spin_limit ? st->spin_limit : kSpinLimit;
  // this row of the block's inverse (zero past the matrix edge), read before any wait
  const T* drow = Dinv + ((size_t)(lower ? 0 : 1) * nb + b) * kSB * kSB + (size_t)rb * kSB;
  T dv[KS];
#pragma unroll
  for (int i = 0; i < KS; ++i) dv[i] = drow[q + KT * i];
  T acc[NC];
#pragma unroll
  for (int cc = 0; cc < NC; ++cc)
    acc[cc] = (q == 0 && live && cc < nrhs) ? In[(long long)row * nrhs + cc] : T(0);
  const T* lrow = LU + (long long)(live ? row : 0) * lda;
  for (int pj = 0; pj < p; ++pj) {
    const int j = lower ? pj : nb - 1 - pj;
    const int c0 = j * kSB;
    T m[KS];                               // issued before the wait: in flight while polling
#pragma unroll
    for (int i = 0; i < KS; ++i) {
      const int col = c0 + q + KT * i;
      m[i] = (live && col < n) ? lrow[col] : T(0);
    }
    if (tid == 0) {
      int ok = 1;
      if (s_front <= (unsigned)pj) {
        unsigned v = 0;
        ok = chain_wait(front, (unsigned)pj + 1, p, err, limit, 1, &v);
        if (ok) s_front = v;
      }
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) return;
    const int kc = min(kSB, n - c0);
    for (int e = tid; e < kSB * nrhs; e += kSolveThreads) {
      const int k = e / nrhs, cc = e - k * nrhs;
      xs[k * kXP + cc] = k < kc ? __ldcg(Out + (long long)(c0 + k) * nrhs + cc) : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < KS; ++i) {
      const T* xr = xs + (q + KT * i) * kXP;
#pragma unroll
      for (int cc = 0; cc < NC; ++cc)
        if (cc < nrhs) acc[cc] = fma(-m[i], xr[cc], acc[cc]);
    }
    __syncthreads();                       // xs is refilled next
  }
  row_sum<KT>(acc, nrhs);                  // y for this row, in every lane of the row
  if (per > 1) {                           // share the chunks' parts of y_b through In
    if (q == 0 && live) {
#pragma unroll
      for (int cc = 0; cc < NC; ++cc)
        if (cc < nrhs) In[(long long)row * nrhs + cc] = acc[cc];
    }
    __syncthreads();
    if (tid == 0) {
      red_release_add(&ready[p], 1u);
      unsigned v = 0;
      s_ok = chain_wait(&ready[p], per, -1, err, limit, 2, &v);
    }
    __syncthreads();
    if (!s_ok) return;
    const int kb = min(kSB, n - b * kSB);
    for (int e = tid; e < kSB * nrhs; e += kSolveThreads) {
      const int k = e / nrhs, cc = e - k * nrhs;
      xs[k * kXP + cc] = k < kb ? __ldcg(In + (long long)(b * kSB + k) * nrhs + cc) : T(0);
    }
  } else if (q == 0) {
#pragma unroll
    for (int cc = 0; cc < NC; ++cc)
      if (cc < nrhs) xs[rb * kXP + cc] = live ? acc[cc] : T(0);
  }
  __syncthreads();
  T xo[NC];
#pragma unroll
  for (int cc = 0; cc < NC; ++cc) xo[cc] = T(0);
#pragma unroll
  for (int i = 0; i < KS; ++i) {
    const T* yr = xs + (q + KT * i) * kXP;
#pragma unroll
    for (int cc = 0; cc < NC; ++cc)
      if (cc < nrhs) xo[cc] = fma(dv[i], yr[cc], xo[cc]);
  }
  row_sum<KT>(xo, nrhs);
  if (q == 0 && live) {
#pragma unroll
    for (int cc = 0; cc < NC; ++cc)
      if (cc < nrhs) Out[(long long)row * nrhs + cc] = xo[cc];
  }
  __syncthreads();
  // x_b's rows are written; the release orders them (cumulatively, through the barrier)
  // before the front moves.  Blocks finish in order, so the front only grows.
  if (tid == 0) {
    if (per == 1) {
      st_release_gpu(front, (unsigned)p + 1);
    } else if (atom_acq_rel_add(&done[p], 1u) == (unsigned)(per - 1)) {
      st_release_gpu(front, (unsigned)p + 1);
    }
  }
}

template <typename T, int RC, int NC>
static cudaError_t trsv_chain_t(const T* LU, long long lda, const T* Dinv, int n, T* In, T* Out, int nrhs,
                                bool lower, unsigned* counters, const DevState* st, cudaStream_t s) {
  const int nb = (n + kSB - 1) / kSB;
  cudaError_t e = cudaMemsetAsync(counters + 1, 0, sizeof(unsigned) * (trsv_counter_words(n) - 1), s);
  if (e != cudaSuccess) return e;
  trsv_chain_kernel<T, RC, NC><<<nb * (kSB / RC), kSolveThreads, 0, s>>>(LU, lda, Dinv, n, In, Out, nrhs,
                                                                           lower ? 1 : 0, counters, st);
  return cudaGetLastError();
}

template <typename T, int RC>
static cudaError_t trsv_chain_nc(const void* LU, long long lda, const void* dinv, int n, void* In, void* Out,
                                 int nrhs, int lower, unsigned* counters, const DevState* st, cudaStream_t s) {
  const T* L = static_cast<const T*>(LU);
  const T* D = static_cast<const T*>(dinv);
  T* I = static_cast<T*>(In);
  T* O = static_cast<T*>(Out);
  if (nrhs == 1) return trsv_chain_t<T, RC, 1>(L, lda, D, n, I, O, nrhs, lower != 0, counters, st, s);
  if (nrhs <= 4) return trsv_chain_t<T, RC, 4>(L, lda, D, n, I, O, nrhs, lower != 0, counters, st, s);
  return trsv_chain_t<T, RC, kXS>(L, lda, D, n, I, O, nrhs, lower != 0, counters, st, s);
}

cudaError_t launch_trsv_chain_selftest(float* scratch, unsigned* counters, const DevState* st, cudaStream_t s) {
  const int n = 128, nb = 2;
  cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(float) * kChainSelftestFloats, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(counters, 0, sizeof(unsigned) * trsv_counter_words(n), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(counters + 1, 1, 1, s);   // the next ticket is 1
  if (e != cudaSuccess) return e;
  float* LU = scratch;
  float* dinv = LU + n * n;
  float* in = dinv + 2 * nb * kSB * kSB;
  trsv_chain_kernel<float, 64, 1><<<1, kSolveThreads, 0, s>>>(LU, n, dinv, n, in, in + n, 1, 1, counters, st);
  return cudaGetLastError();
}

cudaError_t launch_trsv_chain(const void* LU, long long lda, const void* dinv, int n, void* In, void* Out,
                              int nrhs, int lower, int fp32, unsigned* counters, const DevState* st,
                              cudaStream_t s) {
  if (nrhs < 1 || nrhs > kXS || In == Out) return cudaErrorInvalidValue;
  if (n == 0) return cudaSuccess;
  // FP32: one CTA per block (one hop per block on the chain); FP64: 4 CTAs per block, so
  // that the two 64-wide products on the chain are spread over 4 SMs' FP64 pipes
  if (fp32) return trsv_chain_nc<float, 64>(LU, lda, dinv, n, In, Out, nrhs, lower, counters, st, s);
  return trsv_chain_nc<double, 16>(LU, lda, dinv, n, In, Out, nrhs, lower, counters, st, s);
}

cudaError_t launch_invert_diag(const double* LU, long long lda, int n, void* dinv, int fp32, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const dim3 grid((n + kSB - 1) / kSB, 2);
  const size_t smem = sizeof(double) * (2 * kSB * kB1 + kSB);
  cudaError_t e = fp32 ? smem_optin(invert_diag_kernel<float>) : smem_optin(invert_diag_kernel<double>);
  if (e != cudaSuccess) return e;
  if (fp32) invert_diag_kernel<float><<<grid, kSB, smem, s>>>(LU, lda, n, static_cast<float*>(dinv));
  else invert_diag_kernel<double><<<grid, kSB, smem, s>>>(LU, lda, n, static_cast<double*>(dinv));
  return cudaGetLastError();
}

cudaError_t launch_trsv(const void* LU, long long lda, const void* dinv, int n, void* Y, int nrhs, int lower,
                        int fp32, unsigned* counters, cudaStream_t s) {
  if (fp32)
    return trsv_t(static_cast<const float*>(LU), lda, static_cast<const float*>(dinv), n, static_cast<float*>(Y),
                  nrhs, lower != 0, counters, s);
  return trsv_t(static_cast<const double*>(LU), lda, static_cast<const double*>(dinv), n, static_cast<double*>(Y),
                nrhs, lower != 0, counters, s);
}

// FP32 copy of the factors (for the correction solves of the refinement).
__global__ void convert_lu32_kernel(const double* __restrict__ LU, long long lda, int n, float* __restrict__ out) {
  const long long total = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), k = (int)(e - (long long)i * n);
    out[e] = static_cast<float>(LU[(long long)i * lda + k]);
  }
}

cudaError_t launch_convert_lu32(const double* LU, long long lda, int n, float* out, cudaStream_t s) {
  const long long total = (long long)n * n;
  if (total == 0) return cudaSuccess;
  convert_lu32_kernel<<<(int)std::min<long long>((total + 255) / 256, 152 * 16), 256, 0, s>>>(LU, lda, n, out);
  return cudaGetLastError();
}

// Y32 = P B rounded to FP32 (the right-hand side of a correction solve).
__global__ void gather_rows32_kernel(const double* __restrict__ B, long long ldb, const int* __restrict__ perm,
                                     int n, int nrhs, float* __restrict__ Y) {
  const long long total = (long long)n * nrhs;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / nrhs), c = (int)(e - (long long)i * nrhs);
    Y[e] = static_cast<float>(B[(long long)perm[i] * ldb + c]);
  }
}

cudaError_t launch_gather_rows32(const double* B, long long ldb, const int* perm, int n, int nrhs, float* Y,
                                 cudaStream_t s) {
  const long long total = (long long)n * nrhs;
  if (total == 0) return cudaSuccess;
  gather_rows32_kernel<<<(int)std::min<long long>((total + 255) / 256, 152 * 16), 256, 0, s>>>(B, ldb, perm, n,
                                                                                               nrhs, Y);
  return cudaGetLastError();
}

// X += alpha D for an FP32 correction D.
__global__ void axpy_rows32_kernel(double* X, long long ldx, const float* D, double alpha, int n, int nrhs) {
  const long long total = (long long)n * nrhs;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / nrhs), c = (int)(e - (long long)i * nrhs);
    X[(long long)i * ldx + c] = fma(alpha, static_cast<double>(D[e]), X[(long long)i * ldx + c]);
  }
}

cudaError_t launch_axpy_rows32(double* X, long long ldx, const float* D, double alpha, int n, int nrhs,
                               cudaStream_t s) {
  const long long total = (long long)n * nrhs;
  if (total == 0) return cudaSuccess;
  axpy_rows32_kernel<<<(int)std::min<long long>((total + 255) / 256, 152 * 16), 256, 0, s>>>(X, ldx, D, alpha, n,
                                                                                             nrhs);
  return cudaGetLastError();
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
        R[(long long)row * nrhs + c] = B ? B[(long long)row * ldb + c] - ax : ax;   // no B: R = A X
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

// out = max_j sum_i |a_ij| (the matrix 1-norm).  One CTA per 32 columns: warp k sums rows
// k, k + 8, ... of the 32 columns (one coalesced 256-byte row segment per load), the eight
// partial sums are added in a fixed order, and the column maximum is combined by an atomic
// max on the IEEE bits (order-independent), so the result does not depend on scheduling.
__global__ void __launch_bounds__(256) norm1_kernel(const double* __restrict__ A, long long lda, int n,
                                                    double* out) {
  __shared__ double part[8][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = blockIdx.x * 32 + lane;
  double s = 0.0;
  if (col < n)
    for (int i = warp; i < n; i += 8) s += abs_int(A[(long long)i * lda + col]);
  part[warp][lane] = s;
  __syncthreads();
  if (warp == 0) {
    double c = 0.0;
    for (int k = 0; k < 8; ++k) c += part[k][lane];
    unsigned long long b = abs_bits(c);
    for (int off = 16; off > 0; off >>= 1) b = max_bits(b, __shfl_xor_sync(0xffffffffu, b, off));
    if (lane == 0) atomicMax(reinterpret_cast<unsigned long long*>(out), b);
  }
}

cudaError_t launch_norm1(const double* A, long long lda, int n, double* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), s);
  if (e != cudaSuccess || n == 0) return e;
  norm1_kernel<<<(n + 31) / 32, 256, 0, s>>>(A, lda, n, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- GMRES-based refinement
// Krylov vectors are n x nrhs row-major blocks, nrhs independent columns side by side; the
// reductions run in a fixed order, so the refinement's results do not depend on scheduling.

// Y = A X (FP64), one CTA per row.
cudaError_t launch_matvec(const double* A, long long lda, int n, const double* X, long long ldx, int nrhs,
                          double* Y, cudaStream_t s) {
  if (n == 0 || nrhs == 0) return cudaSuccess;
  residual_kernel<<<std::min(n, 152 * 8), kSolveThreads, 0, s>>>(A, lda, n, X, ldx, nrhs, nullptr, 0, Y);
  return cudaGetLastError();
}

// out[i * nrhs + c] = sum_r V_i[r][c] W[r][c] for i < nvec (V_i = V + i * n * nrhs): one CTA
// per i, each thread a fixed stride of rows, then a fixed-order tree per column.
constexpr int kMaxGmresRhs = 16;
__global__ void __launch_bounds__(kSolveThreads) block_dots_kernel(const double* __restrict__ V, int nvec, int n,
                                                                   int nrhs, const double* __restrict__ W,
                                                                   double* __restrict__ out) {
  __shared__ double red[kSolveThreads];
  const int i = blockIdx.x;
  if (i >= nvec) return;
  const double* v = V + (size_t)i * n * nrhs;
  for (int c0 = 0; c0 < nrhs; c0 += kMaxGmresRhs) {
    const int nc = min(kMaxGmresRhs, nrhs - c0);
    double acc[kMaxGmresRhs];
#pragma unroll
    for (int c = 0; c < kMaxGmresRhs; ++c) acc[c] = 0.0;
    for (int r = threadIdx.x; r < n; r += blockDim.x)
#pragma unroll
      for (int c = 0; c < kMaxGmresRhs; ++c)
        if (c < nc) acc[c] = fma(v[(size_t)r * nrhs + c0 + c], W[(size_t)r * nrhs + c0 + c], acc[c]);
#pragma unroll
    for (int c = 0; c < kMaxGmresRhs; ++c) {
      if (c >= nc) break;                            // uniform across the CTA
      __syncthreads();
      red[threadIdx.x] = acc[c];
      __syncthreads();
      for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
      }
      if (threadIdx.x == 0) out[(size_t)i * nrhs + c0 + c] = red[0];
    }
  }
}

cudaError_t launch_block_dots(const double* V, int nvec, int n, int nrhs, const double* W, double* out,
                              cudaStream_t s) {
  if (nvec == 0 || n == 0 || nrhs == 0) return cudaSuccess;
  block_dots_kernel<<<nvec, kSolveThreads, 0, s>>>(V, nvec, n, nrhs, W, out);
  return cudaGetLastError();
}

// W[r][c] += sign * sum_{i < nvec} coef[i * nrhs + c] V_i[r][c]   (i in ascending order)
__global__ void block_axpy_kernel(const double* __restrict__ V, int nvec, int n, int nrhs,
                                  const double* __restrict__ coef, double sign, double* __restrict__ W) {
  const long long total = (long long)n * nrhs;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % nrhs);
    double acc = 0.0;
    for (int i = 0; i < nvec; ++i) acc = fma(coef[(size_t)i * nrhs + c], V[(size_t)i * total + e], acc);
    W[e] = fma(sign, acc, W[e]);
  }
}

cudaError_t launch_block_axpy(const double* V, int nvec, int n, int nrhs, const double* coef, double sign,
                              double* W, cudaStream_t s) {
  const long long total = (long long)n * nrhs;
  if (total == 0 || nvec == 0) return cudaSuccess;
  block_axpy_kernel<<<(int)std::min<long long>((total + 255) / 256, 152 * 16), 256, 0, s>>>(V, nvec, n, nrhs, coef,
                                                                                            sign, W);
  return cudaGetLastError();
}

// Y[r][c] = scale[c] * X[r][c] with X in FP32 or FP64 (x32 != nullptr selects FP32).
__global__ void scale_cols_kernel(const double* __restrict__ X, const float* __restrict__ x32, int n, int nrhs,
                                  const double* __restrict__ scale, double* __restrict__ Y) {
  const long long total = (long long)n * nrhs;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const double x = x32 ? static_cast<double>(x32[e]) : X[e];
    Y[e] = scale ? scale[e % nrhs] * x : x;
  }
}

cudaError_t launch_scale_cols(const double* X, const float* x32, int n, int nrhs, const double* scale, double* Y,
                              cudaStream_t s) {
  const long long total = (long long)n * nrhs;
  if (total == 0) return cudaSuccess;
  scale_cols_kernel<<<(int)std::min<long long>((total + 255) / 256, 152 * 16), 256, 0, s>>>(X, x32, n, nrhs, scale, Y);
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
