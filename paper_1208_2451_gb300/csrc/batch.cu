// Batched LU_PRRP solves of many independent small systems (n <= 1024) in one persistent
// launch: each CTA takes the next system from a size-sorted work list and runs the whole
// of Algorithm 1 on it, then the solve and FP64 iterative refinement (Section 3.3).
//
// Precision (the FP32-factor / FP64-refinement form): the working copy of the matrix is
// stored in T (float, or double for the plain-FP64 batched form); the panel's strong RRQR
// (QR with column pivoting, the tau test and interchanges, Algorithm 2), the diagonal-block
// GEPP and the refinement residual r = b - A x are computed in FP64.  The Schur update,
// U12 and the final multipliers are computed in T.  Substitutions use T's arithmetic on
// the T factors (the refinement residual and solution stay FP64).
//
// Inside a CTA: the panel (m x w, w <= 32) lives in shared memory in FP64; one thread
// works on one panel row; argmax keys compare non-negative doubles by their IEEE bit
// patterns.  The trailing matrix stays in the CTA's global scratch (L2-resident for
// these sizes).  No grid-wide synchronization is used: CTAs never wait on one another.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace prrp {

namespace {

constexpr int kBT = 256;          // threads per batch CTA
constexpr int kBW = 32;           // largest panel width in the batched kernel
constexpr int kUnroll = 4;        // global loads a thread keeps in flight in the copy and update loops
constexpr int kUpd = 8;           // loads a thread keeps in flight in the row moves, and C values a lane
                                  // loads per row before its FMAs in the Schur update
constexpr int kMaxBRows = 4;      // panel rows per thread: the batched entry points refuse n > 1024
static_assert(kMaxBRows * kBT >= 1024, "every panel row has a thread");

struct BKey {
  unsigned long long v;
  int k1, k2;
};

__device__ __forceinline__ bool bbetter(const BKey& a, const BKey& b) {
  if (a.v != b.v) return a.v > b.v;
  if (a.k1 != b.k1) return a.k1 < b.k1;
  return a.k2 < b.k2;
}

__device__ __forceinline__ BKey bshfl(const BKey& c, int m, unsigned mask) {
  BKey o;
  o.v = __shfl_xor_sync(mask, c.v, m);
  o.k1 = __shfl_xor_sync(mask, c.k1, m);
  o.k2 = __shfl_xor_sync(mask, c.k2, m);
  return o;
}

__device__ __forceinline__ unsigned long long dbits(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x));
}

// Block-wide best key, returned to every thread (two __syncthreads).
__device__ BKey block_best_key(BKey c, BKey* s_w) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const BKey o = bshfl(c, off, 0xffffffffu);
    if (bbetter(o, c)) c = o;
  }
  if (lane == 0) s_w[warp] = c;
  __syncthreads();
  BKey r = s_w[0];
  for (int k = 1; k < kBT / 32; ++k)
    if (bbetter(s_w[k], r)) r = s_w[k];
  __syncthreads();
  return r;
}

// Block-wide sums of three values, each returned to every thread (two __syncthreads);
// s_red holds 3 kBT / 32 doubles.
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c, double* s_red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, off);
    b += __shfl_xor_sync(0xffffffffu, b, off);
    c += __shfl_xor_sync(0xffffffffu, c, off);
  }
  if (lane == 0) {
    s_red[warp] = a;
    s_red[kBT / 32 + warp] = b;
    s_red[2 * (kBT / 32) + warp] = c;
  }
  __syncthreads();
  double ra = 0.0, rb = 0.0, rc = 0.0;
  for (int k = 0; k < kBT / 32; ++k) {
    ra += s_red[k];
    rb += s_red[kBT / 32 + k];
    rc += s_red[2 * (kBT / 32) + k];
  }
  __syncthreads();
  a = ra;
  b = rb;
  c = rc;
}

__device__ __forceinline__ double block_max(double v, double* s_red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  if (lane == 0) s_red[warp] = v;
  __syncthreads();
  double r = 0.0;
  for (int k = 0; k < kBT / 32; ++k) r = fmax(r, s_red[k]);
  __syncthreads();
  return r;
}

// Strong RRQR of the transposed m x w panel held in Ps (FP64, stride sp), Algorithm 2.
// On return pos[r] is the final position of panel row r and rows with pos >= w hold their
// multipliers M(:, pos - w) = (R11^-1 R12)(:, .).  Returns 0, or a prrp_status.
// One thread per panel row: an FP64 instruction holds its sub-partition's FP64 unit for
// 64 cycles whatever its active lanes, so whole rows per lane (no team reductions, no
// per-row fixed cost spread over several lanes) issue the fewest FP64 instructions.  For
// the same reason the argmax key and the norm-recompute test compare IEEE bit patterns on
// the integer pipe (non-negative doubles order as their bits), and thr[r] keeps 1e-4 times
// the row's last exactly computed squared norm.
__device__ int batch_panel_select(double* Ps, int sp, int m, int w, double tau, int max_swaps,
                                  double* nrm, double* thr, int* pos, double* Rs, double* rdiag,
                                  BKey* s_w, int* swaps_out) {
  __shared__ double s_refl[3];                   // alpha, beta, v0 of the current reflector
  const int tid = threadIdx.x, lane = tid & 31;
  for (int r = tid; r < m; r += kBT) {
    const double* x = Ps + r * sp;
    double s0 = 0.0, s1 = 0.0;
    int i = 0;
    for (; i + 1 < w; i += 2) { s0 = fma(x[i], x[i], s0); s1 = fma(x[i + 1], x[i + 1], s1); }
    if (i < w) s0 = fma(x[i], x[i], s0);
    const double s = s0 + s1;
    nrm[r] = s; thr[r] = 1e-4 * s; pos[r] = r;
  }
  __syncthreads();
  for (int t = 0; t < w; ++t) {
    BKey c{0ull, 0x7fffffff, 0};
    for (int r = tid; r < m; r += kBT)
      if (pos[r] >= t) {
        // the key of fmax(nrm, 0): negative values and NaN count as 0
        const long long nb = static_cast<long long>(dbits(nrm[r]));
        BKey d{nb > 0 && nb <= static_cast<long long>(kInfBits) ? static_cast<unsigned long long>(nb) : 0ull, pos[r], r};
        if (bbetter(d, c)) c = d;
      }
    // block argmax, then the reflector's scalars formed once and broadcast with the next
    // barrier
    BKey g = c;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const BKey o = bshfl(g, off, 0xffffffffu);
      if (bbetter(o, g)) g = o;
    }
    if (lane == 0) s_w[tid >> 5] = g;
    __syncthreads();
    g = s_w[0];
    for (int k = 1; k < kBT / 32; ++k)
      if (bbetter(s_w[k], g)) g = s_w[k];
    if (g.v == 0ull) return PRRP_ERR_SINGULAR;
    const int rw = g.k2, pw = g.k1;
    const double* xw = Ps + rw * sp;
    // the reflector's scalars (a square root and a division on the FP64 pipe), by the last
    // thread: it owns no panel row while m < kBT, so the rows' partial sums below overlap them
    if (tid == kBT - 1) {
      const double x0 = xw[t];
      const double normx = sqrt(__longlong_as_double(static_cast<long long>(g.v)));
      const double alpha = (x0 >= 0.0) ? -normx : normx;
      s_refl[0] = alpha;
      s_refl[1] = 1.0 / (normx * (normx + abs_int(x0)));
      s_refl[2] = x0 - alpha;
      Rs[t * kBW + t] = alpha;
    }
    // the part of each row's dot product with the reflector that needs no reflector scalar,
    // sum_{i > t} x_w[i] x[i], while those scalars are formed (same arithmetic as below)
    double sdot[kMaxBRows];
#pragma unroll
    for (int q = 0; q < kMaxBRows; ++q) {
      const int r = tid + q * kBT;
      double s1 = 0.0, s2 = 0.0;
      if (r < m && r != rw && pos[r] >= t) {
        const double* x = Ps + r * sp;
        int i = t + 1;
        for (; i + 1 < w; i += 2) { s1 = fma(xw[i], x[i], s1); s2 = fma(xw[i + 1], x[i + 1], s2); }
        if (i < w) s1 = fma(xw[i], x[i], s1);
      }
      sdot[q] = s1 + s2;
    }
    for (int i = tid; i < t; i += kBT) Rs[i * kBW + t] = xw[i];
    __syncthreads();
    const double beta = s_refl[1], v0 = s_refl[2];
    // the winner row's values are read by every thread below; it is itself not updated
#pragma unroll
    for (int q = 0; q < kMaxBRows; ++q) {
      const int r = tid + q * kBT;
      if (r >= m) break;
      const int pr = pos[r];
      if (r == rw) {                                 // the winner takes position t
        pos[r] = t;
        continue;
      }
      if (pr < t) continue;
      double* x = Ps + r * sp;
      const double f = beta * fma(v0, x[t], sdot[q]);
      const double xt = fma(-f, v0, x[t]);
      x[t] = xt;
      for (int k = t + 1; k < w; ++k) x[k] = fma(-f, xw[k], x[k]);
      double n2 = fma(-xt, xt, nrm[r]);
      const long long nb = static_cast<long long>(dbits(n2)), tb = static_cast<long long>(dbits(thr[r]));
      if (!(nb > tb && nb <= static_cast<long long>(kInfBits))) {   // !(n2 > thr): recompute
        double e0 = 0.0, e1 = 0.0;
        int k = t + 1;
        for (; k + 1 < w; k += 2) { e0 = fma(x[k], x[k], e0); e1 = fma(x[k + 1], x[k + 1], e1); }
        if (k < w) e0 = fma(x[k], x[k], e0);
        n2 = e0 + e1;
        thr[r] = 1e-4 * n2;
      }
      nrm[r] = n2;
      pos[r] = (pr == t) ? pw : pr;
    }
    // no barrier here: the next step's argmax reads only this thread's rows, s_w and
    // s_refl were read before the barrier above, and the next winner row's update is
    // ordered by the next step's first barrier
  }
  __syncthreads();
  for (int i = tid; i < w; i += kBT) rdiag[i] = 1.0 / Rs[i * kBW + i];
  __syncthreads();
  for (int r = tid; r < m; r += kBT) {
    if (pos[r] < w) continue;
    double* b = Ps + r * sp;
    for (int i = w - 1; i >= 0; --i) {
      const double mi = b[i] * rdiag[i];
      b[i] = mi;
      for (int k = 0; k < i; ++k) b[k] = fma(-Rs[k * kBW + i], mi, b[k]);
    }
  }
  __syncthreads();
  int swaps = 0;
  for (;;) {
    BKey c{0ull, 0x7fffffff, 0x7fffffff};
    for (int r = tid; r < m; r += kBT) {
      const int pr = pos[r];
      if (pr < w) continue;
      BKey d{0ull, pr - w, 0x7fffffff};
      for (int i = 0; i < w; ++i) {
        const unsigned long long a = abs_bits(Ps[r * sp + i]);
        if (a > d.v || d.k2 == 0x7fffffff) { d.v = a; d.k2 = i; }
      }
      if (bbetter(d, c)) c = d;
    }
    const BKey g = block_best_key(c, s_w);
    if (g.k1 == 0x7fffffff || !(__longlong_as_double(static_cast<long long>(g.v)) > tau)) break;
    if (swaps >= max_swaps) return PRRP_ERR_SWAP_LIMIT;
    const int js = g.k1, is = g.k2;
    // the entering row's column M(:, js), staged before any row changes
    int rin = -1;
    for (int r = tid; r < m; r += kBT)
      if (pos[r] == w + js) rin = r;
    double* colv = rdiag;                                  // reuse: w doubles
    __syncthreads();
    if (rin >= 0)
      for (int i = 0; i < w; ++i) colv[i] = Ps[rin * sp + i];
    __syncthreads();
    const double mu = colv[is];
    for (int r = tid; r < m; r += kBT) {
      const int pr = pos[r];
      double* x = Ps + r * sp;
      if (pr == w + js) {
        pos[r] = is;
      } else if (pr == is) {
        for (int k = 0; k < w; ++k) x[k] = (k == is) ? 1.0 / mu : -colv[k] / mu;
        pos[r] = w + js;
      } else if (pr >= w) {
        const double f = x[is] / mu;
        for (int k = 0; k < w; ++k) x[k] = (k == is) ? f : fma(-f, colv[k], x[k]);
      }
    }
    ++swaps;
    __syncthreads();
  }
  *swaps_out = swaps;
  return 0;
}

template <typename T>
struct BatchArgs {
  int count;
  const int* order;          // systems in processing order (largest first)
  const int* n;
  const double* const* A;    // FP64 input matrices (not modified)
  const int* lda;
  const int* nrhs;
  double* const* B;          // right-hand sides, overwritten by the solutions
  const int* ldb;
  int* const* perm_out;      // optional per-system permutation outputs
  int b;
  double tau;
  int max_swaps;
  int refine_max_iter;
  double refine_target;
  int nmax;
  T* wsW;                    // per CTA: nmax * nmax
  T* wsT;                    // per CTA: tmp_rows * nmax
  int tmp_rows;
  double* wsV;               // per CTA: 5 * nmax doubles
  int* wsI;                  // per CTA: 3 * nmax ints (perm, row moves)
  int* status;               // per system
  int* iters;
  double* eta0;
  double* eta;
  unsigned* counter;         // work list head
};

// sum_k row[k] y_k over one block of the substitution (y_k in Db's spare column), in
// order k = 0, 1, ...: for a full FP32 block every row value is loaded before the first
// FMA, so the loads wait on memory once rather than once per term.
template <typename T>
__device__ __forceinline__ T block_dot(const T* row, int kb, const double* Db) {
  T acc = 0;
  if (sizeof(T) == 4 && kb == 32) {
    T r[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) r[k] = row[k];
#pragma unroll
    for (int k = 0; k < 32; ++k) acc = fma(r[k], static_cast<T>(Db[k * (kBW + 1) + kBW]), acc);
  } else {
    for (int k = 0; k < kb; ++k) acc = fma(row[k], static_cast<T>(Db[k * (kBW + 1) + kBW]), acc);
  }
  return acc;
}

// x[i] -= sum_k W[i][k0 + k] y_k for the rows i in [r0, r1) (y_k in D's spare column).
// FP32: 32 rows per warp pass, lane k reading column k0 + k of every row (one coalesced
// line per row, all 32 loads in flight), and the 32 rows' products summed over the lanes
// by a transposing butterfly (31 shuffles), after which lane r holds row r's sum.  FP64:
// one row per thread (the butterfly's additions would double the FP64 instructions).
template <typename T>
__device__ __forceinline__ void block_rows_update(const T* W, int n, int k0, int kb, const double* D, double* x,
                                                  int r0, int r1) {
  if constexpr (sizeof(T) == 4) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const T yl = lane < kb ? static_cast<T>(D[lane * (kBW + 1) + kBW]) : T(0);
    for (int g0 = r0 + 32 * warp; g0 < r1; g0 += 32 * (kBT / 32)) {
      T v[32];
#pragma unroll
      for (int r = 0; r < 32; ++r)
        v[r] = (lane < kb && g0 + r < r1) ? W[(long long)(g0 + r) * n + k0 + lane] : T(0);
#pragma unroll
      for (int r = 0; r < 32; ++r) v[r] *= yl;
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) {
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int j = 0; j < off; ++j) {
          const T send = up ? v[j] : v[j + off];
          const T keep = up ? v[j + off] : v[j];
          v[j] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
      }
      if (g0 + lane < r1) x[g0 + lane] = static_cast<double>(static_cast<T>(x[g0 + lane]) - v[0]);
    }
  } else {
    for (int i = r0 + threadIdx.x; i < r1; i += kBT)
      x[i] = static_cast<double>(static_cast<T>(x[i]) - block_dot<T>(W + (long long)i * n + k0, kb, D));
  }
}

constexpr int kDb = kBW * (kBW + 1);   // one staged diagonal block: FP64, row stride kBW + 1
static_assert(kUnroll * kBT >= kBW * kBW, "one round of loads stages a whole diagonal block");

// The kb x kb diagonal block at (k0, k0) of W, loaded into registers (kb >= 1) ...
template <typename T>
__device__ __forceinline__ void block_load(const T* W, int n, int k0, int kb, T (&v)[kUnroll]) {
#pragma unroll
  for (int u = 0; u < kUnroll; ++u) {
    const int e = threadIdx.x + u * kBT, i = e / kb, k = e - i * kb;
    v[u] = e < kb * kb ? W[(long long)(k0 + i) * n + k0 + k] : T(0);
  }
}

// ... and stored into Db in FP64.
template <typename T>
__device__ __forceinline__ void block_store(const T (&v)[kUnroll], int kb, double* Db) {
#pragma unroll
  for (int u = 0; u < kUnroll; ++u) {
    const int e = threadIdx.x + u * kBT, i = e / kb, k = e - i * kb;
    if (e < kb * kb) Db[i * (kBW + 1) + k] = static_cast<double>(v[u]);
  }
}

// x (length n, stored in FP64) <- U^-1 L^-1 P y for the T factors in W (ld n); y = b or r
// in v, x out.  The arithmetic is T's: FP32 factors give FP32-accurate solutions whatever
// the arithmetic, so the FP32-factor form solves in FP32 (its refinement keeps the
// residual and the accumulated solution in FP64, Section 3.3); dependent FP64 chains would
// cost 64 cycles per step on this GPU.
// Blocks of 32 rows: warp 0 solves a block's triangle by a chain of shuffles, then every
// thread takes the block's solution out of its rows beyond the block and, in the same
// phase, stages the next block's diagonal into the other half of Db, so a block costs two
// barriers and the staging loads wait on memory together with the update's.  The backward
// chain multiplies by each diagonal's reciprocal, formed by its lane before the chain.
// Db: 2 kDb doubles of shared scratch.  Not inlined: its register needs then stay out of
// the kernel body's allocation, which spilled with it inlined.
template <typename T>
__device__ __noinline__ void batch_lu_solve(const T* W, int n, const int* perm, const double* rhs, double* x, double* Db) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nfwd = (n + 31) / 32;                    // forward blocks [32 q, 32 q + 32)
  T sv[kUnroll];
  for (int i = tid; i < n; i += kBT) x[i] = rhs[perm[i]];
  block_load(W, n, 0, min(32, n), sv);
  block_store(sv, min(32, n), Db);
  __syncthreads();
  int buf = 0;
  // forward substitution
  for (int q = 0; q < nfwd; ++q) {
    const int k0 = 32 * q, kb = min(32, n - k0);
    double* D = Db + buf * kDb;
    if (warp == 0) {
      T y = lane < kb ? static_cast<T>(x[k0 + lane]) : T(0);
#pragma unroll
      for (int k = 0; k < kBW - 1; ++k) {
        const T lk = static_cast<T>(D[lane * (kBW + 1) + k]);   // in the buffer for every lane; used only inside the block
        if (k + 1 < kb) {
          const T xk = __shfl_sync(0xffffffffu, y, k);
          if (lane > k) y = fma(-lk, xk, y);
        }
      }
      if (lane < kb) {
        x[k0 + lane] = static_cast<double>(y);
        D[lane * (kBW + 1) + kBW] = static_cast<double>(y);   // the block's solution, for the rows below
      }
    }
    __syncthreads();
    // the next block's diagonal: the next forward block, after the last one the first
    // backward block [max(0, n - 32), n)
    const int s0 = q + 1 < nfwd ? k0 + 32 : max(0, n - 32);
    const int sb = q + 1 < nfwd ? min(32, n - s0) : n - s0;
    block_load(W, n, s0, sb, sv);
    block_rows_update<T>(W, n, k0, kb, D, x, k0 + kb, n);
    block_store(sv, sb, Db + (buf ^ 1) * kDb);
    __syncthreads();
    buf ^= 1;
  }
  // backward substitution, blocks [max(0, kend - 32), kend)
  for (int kend = n; kend > 0; kend -= 32) {
    const int k0 = max(0, kend - 32), kb = kend - k0;
    double* D = Db + buf * kDb;
    if (warp == 0) {
      T y = lane < kb ? static_cast<T>(x[k0 + lane]) : T(0);
      const T rinv = lane < kb ? T(1) / static_cast<T>(D[lane * (kBW + 1) + lane]) : T(0);
#pragma unroll
      for (int k = kBW - 1; k >= 0; --k) {
        const T uk = static_cast<T>(D[lane * (kBW + 1) + k]);   // in the buffer for every lane; used only inside the block
        if (k < kb) {
          if (lane == k) y *= rinv;
          const T xk = __shfl_sync(0xffffffffu, y, k);
          if (lane < k) y = fma(-uk, xk, y);
        }
      }
      if (lane < kb) {
        x[k0 + lane] = static_cast<double>(y);
        D[lane * (kBW + 1) + kBW] = static_cast<double>(y);   // the block's solution, for the rows above
      }
    }
    __syncthreads();
    const int s0 = max(0, k0 - 32), sb = k0 - s0;
    if (sb > 0) block_load(W, n, s0, sb, sv);
    block_rows_update<T>(W, n, k0, kb, D, x, 0, k0);
    if (sb > 0) block_store(sv, sb, Db + (buf ^ 1) * kDb);
    __syncthreads();
    buf ^= 1;
  }
}

// RB: the Schur update's register tile, RB rows of L21 per warp pass (each staged value of
// A12 feeds RB FMAs); chosen per workload by the autotuner together with CTAs per SM (FP32
// working copies only: two FP64 rows of up to 32 multipliers exceed the register budget).
// WB: the panel widths this instantiation serves (w <= WB; 16 or kBW), the length of the
// per-thread register arrays of the update, U12 and the final multipliers.
template <typename T, int RB, int WB>
__global__ void __launch_bounds__(kBT, 2) batch_kernel(BatchArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ BKey s_w[kBT / 32];
  __shared__ double s_red[3 * (kBT / 32)];
  __shared__ int s_sys, s_status, s_np;
  __shared__ double s_rp;                           // reciprocal of the current GEPP pivot
  __shared__ double Rs[kBW * kBW];
  __shared__ double rdiag[kBW];
  __shared__ int ipiv[kBW];
  __shared__ int s_src[kBW];                        // GEPP's interchanges composed: position <- row
  __shared__ double Dg[kBW * (kBW + 1)];
  __shared__ T Lt[kBW * (kBW + 1)];                 // L11 in T, for U12 and the final multipliers
  const int tid = threadIdx.x;
  T* W = a.wsW + (size_t)blockIdx.x * a.nmax * a.nmax;
  T* Tmp = a.wsT + (size_t)blockIdx.x * a.tmp_rows * a.nmax;
  double* V = a.wsV + (size_t)blockIdx.x * 5 * a.nmax;
  int* perm = a.wsI + (size_t)blockIdx.x * 3 * a.nmax;
  int* mv = perm + a.nmax;                          // row moves (dst, src) of one panel: <= 2m ints

  for (;;) {
    if (tid == 0) s_sys = static_cast<int>(atomicAdd(a.counter, 1u));
    __syncthreads();
    const int qi = s_sys;
    if (qi >= a.count) return;
    const int sys = a.order[qi];
    const int n = a.n[sys], lda = a.lda[sys];
    const double* A = a.A[sys];
    if (tid == 0) s_status = 0;
    int swaps_total = 0;
    // ---- working copy and permutation
    {
      const long long nn = (long long)n * n;
      bool bad = false;
      for (long long e0 = tid; e0 < nn; e0 += kUnroll * kBT) {   // kUnroll loads in flight
        double v[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const long long e = e0 + (long long)u * kBT;
          const int i = static_cast<int>(e / n), j = static_cast<int>(e - (long long)i * n);
          v[u] = e < nn ? A[(long long)i * lda + j] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const long long e = e0 + (long long)u * kBT;
          if (e < nn) {
            bad |= abs_bits(v[u]) >= kInfBits;
            W[e] = static_cast<T>(v[u]);
          }
        }
      }
      if (bad) s_status = PRRP_ERR_NONFINITE;
    }
    for (int i = tid; i < n; i += kBT) perm[i] = i;
    __syncthreads();
    // ---- Algorithm 1
    for (int k0 = 0; k0 < n && s_status == 0; k0 += a.b) {
      const int w = min(a.b, n - k0), m = n - k0;
      const int sp = w + 1;
      double* Ps = reinterpret_cast<double*>(smem_raw);
      double* nrm = Ps + (size_t)m * sp;
      double* thr = nrm + m;
      int* pos = reinterpret_cast<int*>(thr + m);
      for (int e0 = tid; e0 < m * w; e0 += kUnroll * kBT) {
        T v[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const int e = e0 + u * kBT, r = e / w, c = e - r * w;
          v[u] = e < m * w ? W[(long long)(k0 + r) * n + k0 + c] : T(0);
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const int e = e0 + u * kBT, r = e / w, c = e - r * w;
          if (e < m * w) Ps[r * sp + c] = static_cast<double>(v[u]);
        }
      }
      __syncthreads();
      int sw = 0;
      const int st = batch_panel_select(Ps, sp, m, w, a.tau, a.max_swaps, nrm, thr, pos, Rs, rdiag,
                                        s_w, &sw);
      if (st != 0) {
        if (tid == 0) s_status = st;
        __syncthreads();
        break;
      }
      swaps_total += sw;
      // row moves: positions that changed, staged whole through Tmp (all n columns)
      if (tid == 0) s_np = 0;
      __syncthreads();
      for (int r = tid; r < m; r += kBT)
        if (pos[r] != r) {
          const int k = atomicAdd(&s_np, 1);
          mv[2 * k] = pos[r];
          mv[2 * k + 1] = r;
        }
      __syncthreads();
      const int np = s_np;
      // every source row is read before any destination is written: np <= 2 (w + swaps)
      // and np <= m, and Tmp holds min(nmax, 2 (b + max_swaps) + 2) rows
      if (np > a.tmp_rows) {
        if (tid == 0) s_status = PRRP_ERR_UNSUPPORTED;
        __syncthreads();
        break;
      }
      for (int e0 = tid; e0 < np * n; e0 += kUpd * kBT) {
        T v[kUpd];
#pragma unroll
        for (int u = 0; u < kUpd; ++u) {
          const int e = e0 + u * kBT, k = e / n, j = e - k * n;
          v[u] = e < np * n ? W[(long long)(k0 + mv[2 * k + 1]) * n + j] : T(0);
        }
#pragma unroll
        for (int u = 0; u < kUpd; ++u) {
          const int e = e0 + u * kBT;
          if (e < np * n) Tmp[e] = v[u];
        }
      }
      __syncthreads();
      for (int e0 = tid; e0 < np * n; e0 += kUpd * kBT) {
        T v[kUpd];
#pragma unroll
        for (int u = 0; u < kUpd; ++u) {
          const int e = e0 + u * kBT;
          v[u] = e < np * n ? Tmp[e] : T(0);
        }
#pragma unroll
        for (int u = 0; u < kUpd; ++u) {
          const int e = e0 + u * kBT, k = e / n, j = e - k * n;
          if (e < np * n) W[(long long)(k0 + mv[2 * k]) * n + j] = v[u];
        }
      }
      __syncthreads();
      // perm follows the same moves: every moved row's id is read before any is written
      for (int k = tid; k < np; k += kBT) mv[2 * k + 1] = perm[k0 + mv[2 * k + 1]];
      __syncthreads();
      for (int k = tid; k < np; k += kBT) perm[k0 + mv[2 * k]] = mv[2 * k + 1];
      // block multipliers L21 into the strip of the rows below the block
      for (int e = tid; e < m * w; e += kBT) {
        const int r = e / w, c = e - r * w;
        const int pr = pos[r];
        if (pr >= w) W[(long long)(k0 + pr) * n + k0 + c] = static_cast<T>(Ps[r * sp + c]);
      }
      __syncthreads();
      // Schur update A22 -= L21 A12 in T: A12 (w x nc) staged in shared memory (the
      // panel's space is free now), one warp per row of L21 (held in registers), lanes
      // along the columns
      const int nc = n - k0 - w;
      T* Us = reinterpret_cast<T*>(smem_raw);
      for (int e0 = tid; e0 < w * nc; e0 += kUnroll * kBT) {
        T v[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const int e = e0 + u * kBT, k = e / max(nc, 1), j = e - k * nc;
          v[u] = e < w * nc ? W[(long long)(k0 + k) * n + k0 + w + j] : T(0);
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const int e = e0 + u * kBT;
          if (e < w * nc) Us[e] = v[u];
        }
      }
      __syncthreads();
      {
        const int lane = tid & 31, warp = tid >> 5;
        const int rows = m - w;
        for (int i0 = warp * RB; i0 < rows; i0 += (kBT / 32) * RB) {
          T lr[RB][WB];
#pragma unroll
          for (int r = 0; r < RB; ++r) {
            const T* l = W + (long long)(k0 + w + i0 + r) * n + k0;
#pragma unroll
            for (int k = 0; k < WB; ++k) lr[r][k] = (k < w && i0 + r < rows) ? l[k] : T(0);
          }
          for (int j0 = lane; j0 < nc; j0 += 32 * kUpd) {
            T cv[RB][kUpd];                       // the C values, loaded before any use
#pragma unroll
            for (int u = 0; u < kUpd; ++u)
#pragma unroll
              for (int r = 0; r < RB; ++r) {
                const int j = j0 + 32 * u;
                cv[r][u] = (j < nc && i0 + r < rows) ? W[(long long)(k0 + w + i0 + r) * n + k0 + w + j] : T(0);
              }
#pragma unroll
            for (int u = 0; u < kUpd; ++u) {
              const int j = j0 + 32 * u;
              if (j >= nc) break;
              T acc[RB];
#pragma unroll
              for (int r = 0; r < RB; ++r) acc[r] = 0;
#pragma unroll
              for (int k = 0; k < WB; ++k)
                if (k < w) {
                  const T uk = Us[k * nc + j];
#pragma unroll
                  for (int r = 0; r < RB; ++r) acc[r] = fma(lr[r][k], uk, acc[r]);
                }
#pragma unroll
              for (int r = 0; r < RB; ++r)
                if (i0 + r < rows) W[(long long)(k0 + w + i0 + r) * n + k0 + w + j] = cv[r][u] - acc[r];
            }
          }
        }
      }
      __syncthreads();
      // GEPP on the diagonal block in FP64
      for (int e = tid; e < w * w; e += kBT) {
        const int i = e / w, j = e - i * w;
        Dg[i * (kBW + 1) + j] = static_cast<double>(W[(long long)(k0 + i) * n + k0 + j]);
      }
      __syncthreads();
      for (int t = 0; t < w; ++t) {
        if (tid == 0) {
          int p = t;
          unsigned long long bv = abs_bits(Dg[t * (kBW + 1) + t]);
          for (int i = t + 1; i < w; ++i) {
            const unsigned long long v = abs_bits(Dg[i * (kBW + 1) + t]);
            if (v > bv) { bv = v; p = i; }
          }
          ipiv[t] = bv > 0ull ? p : -1;
          s_rp = bv > 0ull ? 1.0 / Dg[p * (kBW + 1) + t] : 0.0;   // once for the CTA
        }
        __syncthreads();
        const int p = ipiv[t];
        if (p < 0) {                                   // zero pivot in the diagonal block
          if (tid == 0) s_status = PRRP_ERR_SINGULAR;
          break;
        }
        if (p != t)
          for (int j = tid; j < w; j += kBT) {
            const double x = Dg[t * (kBW + 1) + j];
            Dg[t * (kBW + 1) + j] = Dg[p * (kBW + 1) + j];
            Dg[p * (kBW + 1) + j] = x;
          }
        __syncthreads();
        const double rp = s_rp;
        for (int e = tid; e < (w - t - 1) * (w - t); e += kBT) {
          const int i = t + 1 + e / (w - t), j = t + e % (w - t);
          const double l = Dg[i * (kBW + 1) + t] * rp;
          if (j > t) Dg[i * (kBW + 1) + j] = fma(-l, Dg[t * (kBW + 1) + j], Dg[i * (kBW + 1) + j]);
        }
        __syncthreads();
        for (int i = t + 1 + tid; i < w; i += kBT) Dg[i * (kBW + 1) + t] *= rp;
        __syncthreads();
      }
      __syncthreads();
      if (s_status != 0) break;
      for (int e = tid; e < w * w; e += kBT) {
        const int i = e / w, j = e - i * w;
        W[(long long)(k0 + i) * n + k0 + j] = static_cast<T>(Dg[i * (kBW + 1) + j]);
      }
      __syncthreads();
      if (tid == 0) {                          // GEPP's interchanges composed: position <- row
        for (int t = 0; t < w; ++t) s_src[t] = t;
        for (int t = 0; t < w; ++t) {
          const int p = ipiv[t];
          if (p != t) { const int y = s_src[t]; s_src[t] = s_src[p]; s_src[p] = y; }
        }
      }
      for (int e = tid; e < w * w; e += kBT) {
        const int i = e / w, k = e - i * w;
        Lt[i * (kBW + 1) + k] = static_cast<T>(Dg[i * (kBW + 1) + k]);
      }
      __syncthreads();
      {                                        // perm follows them, all rows read first
        const int pv = tid < w ? perm[k0 + s_src[tid]] : 0;
        __syncthreads();
        if (tid < w) perm[k0 + tid] = pv;
      }
      // block-row interchanges outside the block and U12 = L11^-1 A12 in T, one column per
      // thread: the column's w values are loaded in their interchanged order into registers
      for (int j = tid; j < n; j += kBT) {
        if (j >= k0 && j < k0 + w) continue;
        T x[WB];
#pragma unroll
        for (int t = 0; t < WB; ++t)
          if (t < w) x[t] = W[(long long)(k0 + s_src[t]) * n + j];
        if (j >= k0 + w) {
#pragma unroll
          for (int k = 0; k < WB; ++k)
            if (k < w) {
#pragma unroll
              for (int i = k + 1; i < WB; ++i)
                if (i < w) x[i] = fma(-Lt[i * (kBW + 1) + k], x[k], x[i]);
            }
        }
#pragma unroll
        for (int t = 0; t < WB; ++t)
          if (t < w) W[(long long)(k0 + t) * n + j] = x[t];
      }
      // final multipliers of the rows below: (L21 with GEPP's column interchanges) * L11 in T,
      // one row per thread in registers
      for (int r = k0 + w + tid; r < n; r += kBT) {
        T* row = W + (long long)r * n + k0;
        T x[WB];
#pragma unroll
        for (int t = 0; t < WB; ++t)
          if (t < w) x[t] = row[s_src[t]];
#pragma unroll
        for (int c = 0; c < WB; ++c)
          if (c < w) {
            T acc = x[c];
#pragma unroll
            for (int i = c + 1; i < WB; ++i)
              if (i < w) acc = fma(x[i], Lt[i * (kBW + 1) + c], acc);
            row[c] = acc;
          }
      }
      __syncthreads();
    }
    __syncthreads();
    const int fstat = s_status;
    if (a.perm_out && a.perm_out[sys] && fstat == 0)
      for (int i = tid; i < n; i += kBT) a.perm_out[sys][i] = perm[i];
    // ---- solve and FP64 refinement, one right-hand side at a time
    double* xv = V;
    double* Db = reinterpret_cast<double*>(smem_raw);   // the substitution's two diagonal blocks (the panel's space)
    double* rv = V + a.nmax;
    double* dv = rv + a.nmax;
    const int nr = a.nrhs[sys], ldb = a.ldb[sys];
    double* Bp = a.B[sys];
    double e0max = 0.0, emax = 0.0;
    int itmax = 0;
    double anorm = 0.0;
    if (fstat == 0) {
      // ||A||_1 only scales eta: FP32 sums (relative error ~n 2^-24) on the FP32 pipe
      // instead of n^2 FP64 additions
      float cm = 0.0f;
      for (int j = tid; j < n; j += kBT) {
        float s0 = 0.0f, s1 = 0.0f;
        int i = 0;
        for (; i + 1 < n; i += 2) {
          s0 += fabsf(static_cast<float>(A[(long long)i * lda + j]));
          s1 += fabsf(static_cast<float>(A[(long long)(i + 1) * lda + j]));
        }
        if (i < n) s0 += fabsf(static_cast<float>(A[(long long)i * lda + j]));
        cm = fmaxf(cm, s0 + s1);
      }
      anorm = block_max(static_cast<double>(cm), s_red);
    }
    for (int c = 0; c < nr && fstat == 0; ++c) {
      double* bcol = dv;                                   // the right-hand side, packed
      for (int i = tid; i < n; i += kBT) bcol[i] = Bp[(long long)i * ldb + c];
      __syncthreads();
      batch_lu_solve<T>(W, n, perm, bcol, xv, Db);
      double eta = 0.0, eta_first = 0.0;
      int it = 0;
      for (;;) {
        // r = b - A x in FP64 and eta = ||r||_1 / (||A||_1 ||x||_1 + ||b||_1).  Four rows per
        // warp pass, lanes along the columns (coalesced, four independent FMA chains per
        // lane); the four rows' lane sums are reduced together by a transposing butterfly
        // (lanes 16..31 keep rows 2, 3 and lanes 0..15 rows 0, 1; then the lanes with bit 3
        // set keep the odd row), six FP64 additions for four rows instead of twenty.
        double rs = 0.0, xs = 0.0, bs = 0.0;
        const int lane = tid & 31, warp = tid >> 5;
        const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0;
        const int qr = (h16 ? 2 : 0) + (h8 ? 1 : 0);     // the row this lane's sum ends in
        for (int i0 = 4 * warp; i0 < n; i0 += 4 * (kBT / 32)) {
          const int nrow = min(4, n - i0);
          double acc[4] = {0.0, 0.0, 0.0, 0.0};
          for (int k = lane; k < n; k += 32) {
            const double xk = xv[k];
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (q < nrow) acc[q] = fma(A[(long long)(i0 + q) * lda + k], xk, acc[q]);
          }
          double k0v = h16 ? acc[2] : acc[0], k1v = h16 ? acc[3] : acc[1];
          k0v += __shfl_xor_sync(0xffffffffu, h16 ? acc[0] : acc[2], 16);
          k1v += __shfl_xor_sync(0xffffffffu, h16 ? acc[1] : acc[3], 16);
          double c = h8 ? k1v : k0v;
          c += __shfl_xor_sync(0xffffffffu, h8 ? k0v : k1v, 8);
          c += __shfl_xor_sync(0xffffffffu, c, 4);
          c += __shfl_xor_sync(0xffffffffu, c, 2);
          c += __shfl_xor_sync(0xffffffffu, c, 1);
          if ((lane & 7) == 0 && qr < nrow) {
            const double r = bcol[i0 + qr] - c;
            rv[i0 + qr] = r;
            rs += abs_int(r);
          }
        }
        for (int i = tid; i < n; i += kBT) {
          xs += abs_int(xv[i]);
          bs += abs_int(bcol[i]);
        }
        block_sum3(rs, xs, bs, s_red);
        const double den = anorm * xs + bs;
        const double e = den > 0.0 ? rs / den : (rs > 0.0 ? INFINITY : 0.0);
        if (it == 0) eta_first = e;
        if (it > 0 && e > eta / 2) {                      // stagnation: keep the better
          if (e > eta)
            for (int i = tid; i < n; i += kBT) xv[i] -= V[4 * a.nmax + i];
          else
            eta = e;
          __syncthreads();
          break;
        }
        eta = e;
        if (eta <= a.refine_target || it >= a.refine_max_iter) break;
        double* corr = V + 4 * a.nmax;
        double* rhs_r = V + 3 * a.nmax;
        for (int i = tid; i < n; i += kBT) rhs_r[i] = rv[i];
        __syncthreads();
        batch_lu_solve<T>(W, n, perm, rhs_r, corr, Db);
        for (int i = tid; i < n; i += kBT) xv[i] += corr[i];
        __syncthreads();
        ++it;
      }
      for (int i = tid; i < n; i += kBT) Bp[(long long)i * ldb + c] = xv[i];
      __syncthreads();
      e0max = fmax(e0max, eta_first);
      emax = fmax(emax, eta);
      itmax = max(itmax, it);
    }
    if (tid == 0) {
      a.status[sys] = fstat;
      a.iters[sys] = itmax;
      a.eta0[sys] = fstat == 0 ? e0max : -1.0;
      a.eta[sys] = fstat == 0 ? emax : -1.0;
    }
    (void)swaps_total;
    __syncthreads();
  }
}

}  // namespace

size_t batch_smem_bytes(int nmax, int b) {
  // the panel (m x (b + 1) doubles, norms, positions), reused by the substitution's two
  // staged diagonal blocks
  const size_t panel = (size_t)nmax * (b + 1) * sizeof(double) + (size_t)nmax * (2 * sizeof(double) + sizeof(int));
  return std::max(panel, (size_t)2 * kDb * sizeof(double)) + 64;
}

cudaError_t launch_batch(int fp64, int grid, int rb, const BatchLaunch& L, cudaStream_t s) {
  const size_t smem = batch_smem_bytes(L.nmax, L.b);
  if (fp64) {
    BatchArgs<double> a{L.count, L.order, L.n, L.A, L.lda, L.nrhs, L.B, L.ldb, L.perm_out, L.b, L.tau, L.max_swaps,
                        L.refine_max_iter, L.refine_target, L.nmax, static_cast<double*>(L.wsW),
                        static_cast<double*>(L.wsT), L.tmp_rows, L.wsV, L.wsI, L.status, L.iters,
                        L.eta0, L.eta, L.counter};
    if (L.b <= 16) batch_kernel<double, 1, 16><<<grid, kBT, smem, s>>>(a);   // one FP64 row of L21 per pass
    else batch_kernel<double, 1, kBW><<<grid, kBT, smem, s>>>(a);
  } else {
    BatchArgs<float> a{L.count, L.order, L.n, L.A, L.lda, L.nrhs, L.B, L.ldb, L.perm_out, L.b, L.tau, L.max_swaps,
                       L.refine_max_iter, L.refine_target, L.nmax, static_cast<float*>(L.wsW),
                       static_cast<float*>(L.wsT), L.tmp_rows, L.wsV, L.wsI, L.status, L.iters,
                       L.eta0, L.eta, L.counter};
    if (L.b <= 16) {
      if (rb == 2) batch_kernel<float, 2, 16><<<grid, kBT, smem, s>>>(a);
      else batch_kernel<float, 1, 16><<<grid, kBT, smem, s>>>(a);
    } else {
      if (rb == 2) batch_kernel<float, 2, kBW><<<grid, kBT, smem, s>>>(a);
      else batch_kernel<float, 1, kBW><<<grid, kBT, smem, s>>>(a);
    }
  }
  return cudaGetLastError();
}

int batch_max_width() { return kBW; }

// Shared-memory opt-in for the batch kernels (outside any stream capture).
cudaError_t prepare_batch(int nmax, int b) {
  (void)nmax;
  (void)b;
  cudaError_t e;
  if ((e = smem_optin(batch_kernel<double, 1, 16>)) != cudaSuccess) return e;
  if ((e = smem_optin(batch_kernel<double, 1, kBW>)) != cudaSuccess) return e;
  if ((e = smem_optin(batch_kernel<float, 1, 16>)) != cudaSuccess) return e;
  if ((e = smem_optin(batch_kernel<float, 1, kBW>)) != cudaSuccess) return e;
  if ((e = smem_optin(batch_kernel<float, 2, 16>)) != cudaSuccess) return e;
  return smem_optin(batch_kernel<float, 2, kBW>);
}

// Synthetic systems for the autotuner: iid entries from a counter hash (Weyl sequence,
// mapped to [-1, 1)), diagonally loaded so every sample is comfortably nonsingular.
__global__ void batch_fill_kernel(double* A, int n, int count, double* B, unsigned seed) {
  const long long total = (long long)count * n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = (unsigned long long)e * 0x9E3779B97F4A7C15ull + seed;
    z ^= z >> 31; z *= 0xBF58476D1CE4E5B9ull; z ^= z >> 29;
    double v = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    const long long r = (e / n) % n, c = e % n;
    if (r == c) v += 4.0;
    A[e] = v;
  }
  const long long tb = (long long)count * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tb;
       e += (long long)gridDim.x * blockDim.x)
    B[e] = 1.0;
}

cudaError_t launch_batch_fill(double* A, int n, int count, double* B, cudaStream_t s) {
  batch_fill_kernel<<<1024, 256, 0, s>>>(A, n, count, B, 12345u);
  return cudaGetLastError();
}

}  // namespace prrp
