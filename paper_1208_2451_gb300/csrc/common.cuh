// Device-side helpers shared by the LU_PRRP kernels: the device state word, a bounded
// grid barrier for co-resident (cooperative) grids, and order-preserving atomics.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "prrp.h"

namespace prrp {

constexpr int kMaxW = 128;              // largest panel width b supported
constexpr int kPanelThreads = 320;      // threads per panel CTA (communication, helper, 8 row warps)
constexpr int kPanelMaxCtas = 160;      // CTAs a panel grid may have (exchange slots per step)
constexpr int kTeam = 4;                // threads cooperating on one panel row
// A bounded wait gives up after this many polls (each poll sleeps ~100 ns): about 1-2 s.
constexpr unsigned kSpinLimit = 1u << 24;

// Lives in device memory; one per context.  Kernels record the first error here and
// every later kernel returns at once when status != 0.
struct DevState {
  int status;                    // prrp_status of the first device-side error
  int info;                      // 1-based column of a zero pivot
  unsigned int barrier;          // grid barrier arrivals (reset before each cooperative launch)
  unsigned int npairs;           // (dst, src) row moves produced by the panel kernel
  int panel_swaps;               // interchanges made by the last panel
  int swaps_total;               // interchanges over the whole factorization
  int panels;                    // panels completed
  int pad;
  unsigned long long gmax_bits;  // max |entry| of A and every block Schur complement (g_W)
  unsigned long long amax_bits;  // max |a_ij| of the input
  unsigned long long l21_bits;   // max |L21|
  unsigned long long umax_bits;  // max |U| (diagonal-block GEPP and U12)
  unsigned int nonfinite;        // set when a NaN/Inf was seen in the input
  unsigned int timeout_site;     // which wait ran out (diagnostic)
  unsigned int spin_limit;       // polls before a wait gives up (0: kSpinLimit)
  unsigned int pad2;
};

// Dynamic shared memory opt-in for a kernel.  The attribute is process-wide, so every
// launcher sets the same value for a given kernel, the most the device allows next to the
// kernel's static shared memory, whatever its own launch needs: concurrent launches from
// several host threads then never see another thread's smaller limit.  Occupancy is
// decided by each launch's actual size.  (227 KB per block on sm_103a.)
constexpr int kSmemOptin = 232448;
cudaError_t smem_optin_ptr(const void* kernel);   // api.cpp: cached per kernel
template <typename F>
inline cudaError_t smem_optin(F* kernel) {
  return smem_optin_ptr(reinterpret_cast<const void*>(kernel));
}

__device__ __forceinline__ int dev_status(const DevState* st) {
  return *((volatile const int*)&st->status);
}

__device__ __forceinline__ void set_error(DevState* st, int code, int info = 0) {
  if (atomicCAS(&st->status, 0, code) == 0 && info) st->info = info;
}

// |x| as its IEEE bit pattern (for x >= 0 the pattern orders like the value), and the
// max of two such patterns.  Both are written in PTX so that they stay integer
// instructions: left to the compiler, the sign-bit mask becomes an FP64 absolute value,
// an instruction on the FP64 pipe, which issues 2 per clock per SM on this GPU.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  unsigned long long r;
  asm("and.b64 %0, %1, 0x7FFFFFFFFFFFFFFF;" : "=l"(r) : "l"(__double_as_longlong(x)));
  return r;
}
__device__ __forceinline__ unsigned long long max_bits(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("max.u64 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
// |x| through the integer path above
__device__ __forceinline__ double abs_int(double x) { return __longlong_as_double(static_cast<long long>(abs_bits(x))); }
constexpr unsigned long long kInfBits = 0x7FF0000000000000ull;   // |x| >= this: inf or nan

// max over non-negative doubles through their IEEE bit patterns (monotone for x >= 0).
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* p, double x) {
  if (!(x >= 0.0)) return;
  atomicMax(p, (unsigned long long)__double_as_longlong(x));
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier for a grid whose CTAs are all co-resident (cooperative launch).
// `target` = (barrier ordinal + 1) * gridDim.x on a counter that starts at 0.
// Returns false (and records PRRP_ERR_TIMEOUT unless another error is already recorded)
// when the wait runs out or another CTA has recorded an error; the caller must return.
__device__ __forceinline__ bool grid_barrier(DevState* st, unsigned target, unsigned site) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&st->barrier, 1u);
    int ok = 1;
    unsigned spins = 0;
    const unsigned limit = st->spin_limit ? st->spin_limit : kSpinLimit;
    while (ld_acquire_u32(&st->barrier) < target) {
      if (dev_status(st) != 0) { ok = 0; break; }
      if (++spins > limit) {
        if (atomicCAS(&st->status, 0, PRRP_ERR_TIMEOUT) == 0) st->timeout_site = site;
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace prrp
