// Device helpers of the strong RRQR selections (Algorithm 2), shared by the LU_PRRP panel
// kernel and the CALU_PRRP tournament kernel so that both decide on the same bits:
// candidate records and their warp-wide argmax, the packed QRCP keys, the Householder
// reflector of a row, row-team sums.  Internal to libprrp.so.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace prrp {
namespace sel {

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
// position.  A key without norm bits (zero norm) is at least kPosMask - (m - 1) > 1, so it
// still beats kNoCand, the key of a CTA without remaining rows; 0 marks an empty slot.
constexpr int kPosBits = 20;
constexpr unsigned long long kPosMask = (1ull << kPosBits) - 1;
constexpr unsigned long long kNoCand = 1ull;
// A key with this bit set beats every key without it (unpivoted QR: the row at position t)
constexpr unsigned long long kTopBit = 1ull << 63;
// the winner's remaining norm is zero: the panel is rank deficient
__device__ __forceinline__ bool key_norm_zero(unsigned long long k) { return ((k & ~kTopBit) >> kPosBits) == 0ull; }
__device__ __forceinline__ unsigned long long qrcp_key(double nrm, int pos) {
  const long long b = __double_as_longlong(nrm);
  return (static_cast<unsigned long long>(b < 0 ? 0 : b) & ~kPosMask) | (kPosMask - static_cast<unsigned>(pos));
}
__device__ __forceinline__ int key_pos(unsigned long long k) { return static_cast<int>(kPosMask - (k & kPosMask)); }

// The largest key of a full warp with the payload of its lane (keys are unique or equal to
// kNoCand / 0, where any lane's payload will do).
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

// The reflector of x = B(t:w, row) from its first entry x0 and ||x||^2:
// H = I - beta v v^T, H x = alpha e_1, v = x - alpha e_1, v^T v = 2 ||x|| (||x|| + |x0|).
__device__ __forceinline__ void reflector(double x0, double nrm2, double* alpha, double* beta) {
  const double normx = sqrt(nrm2);
  *alpha = (x0 >= 0.0) ? -normx : normx;
  *beta = 1.0 / (normx * (normx + abs_int(x0)));
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

}  // namespace sel
}  // namespace prrp
