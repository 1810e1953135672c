// Schur update A22 -= L21 A12 (Algorithm 1, line 7) on the tcgen05 tensor cores, for the
// mixed-precision forms: TF32 (one product) or a 3-term BF16 split (x = hi + mid + lo,
// six products hi*hi + hi*mid + mid*hi + hi*lo + lo*hi + mid*mid, about FP32 accuracy).
// Accumulation is FP32 in tensor memory; the FP64 trailing matrix is updated in the
// epilogue (C_ij -= acc_ij in FP64).
//
// Per 128 x 128 output tile (one CTA, 4 warps):
//   * thread 0 issues TMA loads of every operand slice (K-major, 128-byte swizzled rows,
//     zero-padded to multiples of 128 rows and 64 k) onto one mbarrier, then the
//     tcgen05.mma instructions (M = 128, N = 128, K = 32 bytes each) into a 128-column
//     TMEM accumulator and commits them to a second mbarrier;
//   * the 4 warps read TMEM rows (warp w owns lanes 32w..32w+31), transpose each 32 x 32
//     block through shared memory and update C with row-contiguous, coalesced FP64 loads
//     and stores, tracking max |C| for the growth factor.
// Two CTAs fit per SM, so one CTA's epilogue (HBM-bound) overlaps the other's loads and
// MMAs.  Every wait is bounded: on expiry the CTA records PRRP_ERR_TIMEOUT, waits again
// (bounded) for its own copies, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace prrp {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity, giving up after ~1 s of SM clock.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > 2000000000LL) return false;
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// K-major operand tile with 128-byte swizzle: rows of 128 B, 8-row atoms 1024 B apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);   // start address
  d |= static_cast<uint64_t>(1) << 16;                   // leading byte offset (unused here)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;           // stride byte offset: 8 rows x 128 B
  d |= static_cast<uint64_t>(1) << 46;                   // descriptor version for tcgen05
  d |= static_cast<uint64_t>(2) << 61;                   // 128-byte swizzle
  return d;
}

// Instruction descriptor: FP32 accumulator, A/B format fmt (BF16 = 1 under kind::f16,
// TF32 = 2 under kind::tf32), both K-major, shape M x N.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt, int M, int N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

template <int MODE>
__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                     uint32_t accum) {
  if constexpr (MODE == 0) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
  }
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

constexpr int kBM = 128, kBN = 128, kTmemCols = 128;
constexpr int kStage = 33;   // padded row of the 32 x 32 transpose stage (floats)

template <int MODE>
struct TcCfg {
  static constexpr int EB = MODE == 0 ? 4 : 2;         // operand bytes per element
  static constexpr int CH = MODE == 0 ? 2 : 1;         // 128-byte chunks per 64-wide k block
  static constexpr int NS = MODE == 0 ? 1 : 3;         // slices per operand
  static constexpr int NP = MODE == 0 ? 1 : 6;         // slice products
  static constexpr int TILE_A = kBM * 128;             // bytes per slice-chunk
  static constexpr int TILE_B = kBN * 128;
  static constexpr int OPER_BYTES = NS * CH * (TILE_A + TILE_B);
  static constexpr int SMEM = OPER_BYTES + 4 * 32 * kStage * 4 + 1024;
  static constexpr uint32_t IDESC = make_idesc(MODE == 0 ? 2u : 1u, kBM, kBN);
};

__constant__ int c_prod_a[6] = {0, 0, 1, 0, 2, 1};
__constant__ int c_prod_b[6] = {0, 1, 0, 2, 0, 1};

template <int MODE>
__global__ void __launch_bounds__(128, 1) tc_update_kernel(const __grid_constant__ CUtensorMap tmA,
                                                           const __grid_constant__ CUtensorMap tmB,
                                                           int M, int N, int kblocks, int Mpad, int Npad,
                                                           double* __restrict__ C, long long ldc,
                                                           DevState* st, int track) {
  using Cfg = TcCfg<MODE>;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bar_tma, bar_mma;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  if (dev_status(st) != 0) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = base;
  uint8_t* sB = base + Cfg::NS * Cfg::CH * Cfg::TILE_A;
  float* stage = reinterpret_cast<float*>(base + Cfg::OPER_BYTES) + warp * 32 * kStage;
  const int bm = blockIdx.y * kBM, bn = blockIdx.x * kBN;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&bar_tma, 1);
    mbar_init(&bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  for (int kb = 0; kb < kblocks; ++kb) {
    if (tid == 0 && !s_fail) {
      mbar_expect_tx(&bar_tma, Cfg::OPER_BYTES);
      for (int s = 0; s < Cfg::NS; ++s)
        for (int c = 0; c < Cfg::CH; ++c) {
          const int x = kb * 64 + c * (128 / Cfg::EB);
          tma_load_2d(sA + (s * Cfg::CH + c) * Cfg::TILE_A, &tmA, x, s * Mpad + bm, &bar_tma);
          tma_load_2d(sB + (s * Cfg::CH + c) * Cfg::TILE_B, &tmB, x, s * Npad + bn, &bar_tma);
        }
      if (!mbar_wait_bounded(&bar_tma, kb & 1)) {
        s_fail = 1;
        mbar_wait_bounded(&bar_tma, kb & 1);            // let copies still in flight land
      } else {
        tc_fence_after();
        for (int p = 0; p < Cfg::NP; ++p) {
          const int as = c_prod_a[p], bs = c_prod_b[p];
          for (int c = 0; c < Cfg::CH; ++c) {
            const uint64_t ad = sw128_desc(smem_u32(sA + (as * Cfg::CH + c) * Cfg::TILE_A));
            const uint64_t bd = sw128_desc(smem_u32(sB + (bs * Cfg::CH + c) * Cfg::TILE_B));
#pragma unroll
            for (int k = 0; k < 4; ++k)   // 4 MMAs of 32 bytes of k per 128-byte row
              umma<MODE>(tmem, ad + 2 * k, bd + 2 * k, Cfg::IDESC, (kb | p | c | k) != 0);
          }
        }
        umma_commit(&bar_mma);
        if (!mbar_wait_bounded(&bar_mma, kb & 1)) s_fail = 1;
      }
    }
    __syncthreads();
    if (s_fail) break;
  }
  if (!s_fail) {
    // every thread observes the accumulator's completion before reading tensor memory
    if (!mbar_wait_bounded(&bar_mma, (kblocks - 1) & 1)) s_fail = 1;
  }
  tc_fence_after();
  double cmax = 0.0;
  if (!s_fail) {
    const int rbase = bm + warp * 32;
    for (int c0 = 0; c0 < kBN; c0 += 32) {
      uint32_t r[32];
      tmem_ld32(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0, r);
#pragma unroll
      for (int j = 0; j < 32; ++j) stage[lane * kStage + j] = __uint_as_float(r[j]);
      __syncwarp();
      const int col = bn + c0 + lane;
      const int nrows = min(32, M - rbase);
      if (col < N && nrows > 0) {
        double* cp = C + static_cast<long long>(rbase) * ldc + col;
        double cv[32];
        // issue all loads of this lane's column strip before any store (memory-level
        // parallelism: 32 independent coalesced row loads per warp instruction stream)
#pragma unroll
        for (int rr = 0; rr < 32; ++rr)
          if (rr < nrows) cv[rr] = __ldcs(cp + static_cast<long long>(rr) * ldc);
#pragma unroll
        for (int rr = 0; rr < 32; ++rr)
          if (rr < nrows) {
            const double v = cv[rr] - static_cast<double>(stage[rr * kStage + lane]);
            __stcs(cp + static_cast<long long>(rr) * ldc, v);
            cmax = fmax(cmax, fabs(v));
          }
      }
      __syncwarp();
    }
  } else if (tid == 0) {
    set_error(st, PRRP_ERR_TIMEOUT);
  }
  if (track) {
    for (int off = 16; off > 0; off >>= 1) cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, off));
    if (lane == 0) atomic_max_nonneg(&st->gmax_bits, cmax);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// ---- operand preparation: FP64 -> slices, K-major, zero padded ----
__device__ __forceinline__ uint32_t to_tf32_bits(double x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(static_cast<float>(x)));
  return r;
}

// dst[s][r][k] (rows_pad x kpad each) from element (r, k) of the source, which is
// src[r * ld + k] (rows layout) or src[k * ld + r] (columns layout, i.e. the transpose).
template <int MODE, bool COLS>
__global__ void split_kernel(const double* __restrict__ src, long long ld, int rows, int K, int rows_pad,
                             int kpad, void* __restrict__ dst) {
  const long long total = static_cast<long long>(rows_pad) * kpad;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    int r, k;
    if (COLS) { k = static_cast<int>(e / rows_pad); r = static_cast<int>(e - static_cast<long long>(k) * rows_pad); }
    else      { r = static_cast<int>(e / kpad);     k = static_cast<int>(e - static_cast<long long>(r) * kpad); }
    double x = 0.0;
    if (r < rows && k < K) x = COLS ? src[static_cast<long long>(k) * ld + r] : src[static_cast<long long>(r) * ld + k];
    const long long o = static_cast<long long>(r) * kpad + k;
    if constexpr (MODE == 0) {
      static_cast<uint32_t*>(dst)[o] = to_tf32_bits(x);
    } else {
      __nv_bfloat16* d = static_cast<__nv_bfloat16*>(dst);
      const __nv_bfloat16 hi = __double2bfloat16(x);
      const double r1 = x - static_cast<double>(__bfloat162float(hi));
      const __nv_bfloat16 mid = __double2bfloat16(r1);
      const double r2 = r1 - static_cast<double>(__bfloat162float(mid));
      const __nv_bfloat16 lo = __double2bfloat16(r2);
      d[o] = hi;
      d[total + o] = mid;
      d[2 * total + o] = lo;
    }
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2-D map over a [slices * rows_pad] x kpad row-major operand, box = 128 bytes x 128 rows.
bool make_map(CUtensorMap* m, void* base, int mode, int rows_total, int kpad) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const int eb = mode == 0 ? 4 : 2;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(kpad), static_cast<cuuint64_t>(rows_total)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(kpad) * eb};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(128 / eb), 128};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, mode == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base,
                  dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int MODE>
cudaError_t launch_tc_mode(int M, int N, int K, const double* L, long long ldl, const double* U, long long ldu,
                           double* C, long long ldc, DevState* st, int track, void* wsA, void* wsB,
                           cudaStream_t s) {
  using Cfg = TcCfg<MODE>;
  const int kblocks = (K + 63) / 64, kpad = kblocks * 64;
  const int Mpad = (M + kBM - 1) / kBM * kBM, Npad = (N + kBN - 1) / kBN * kBN;
  const long long ta = static_cast<long long>(Mpad) * kpad, tb = static_cast<long long>(Npad) * kpad;
  split_kernel<MODE, false><<<static_cast<int>(std::min<long long>((ta + 255) / 256, 152 * 16)), 256, 0, s>>>(
      L, ldl, M, K, Mpad, kpad, wsA);
  split_kernel<MODE, true><<<static_cast<int>(std::min<long long>((tb + 255) / 256, 152 * 16)), 256, 0, s>>>(
      U, ldu, N, K, Npad, kpad, wsB);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  CUtensorMap ma, mb;
  if (!make_map(&ma, wsA, MODE, Cfg::NS * Mpad, kpad) || !make_map(&mb, wsB, MODE, Cfg::NS * Npad, kpad))
    return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(tc_update_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
  if (e != cudaSuccess) return e;
  dim3 grid(Npad / kBN, Mpad / kBM);
  tc_update_kernel<MODE><<<grid, 128, Cfg::SMEM, s>>>(ma, mb, M, N, kblocks, Mpad, Npad, C, ldc, st, track);
  return cudaGetLastError();
}

}  // namespace

size_t tc_workspace_bytes(int prec, int M, int N, int K) {
  const int mode = prec == PRRP_TF32 ? 0 : 1;
  const int ns = mode == 0 ? 1 : 3, eb = mode == 0 ? 4 : 2;
  const size_t kpad = static_cast<size_t>((K + 63) / 64) * 64;
  const size_t Mpad = static_cast<size_t>((M + kBM - 1) / kBM) * kBM;
  const size_t Npad = static_cast<size_t>((N + kBN - 1) / kBN) * kBN;
  return ns * eb * kpad * (Mpad + Npad) + 2048;
}

cudaError_t launch_tc_update(int prec, int M, int N, int K, const double* L, long long ldl, const double* U,
                             long long ldu, double* C, long long ldc, DevState* st, int track, void* ws,
                             cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  const int mode = prec == PRRP_TF32 ? 0 : 1;
  const int ns = mode == 0 ? 1 : 3, eb = mode == 0 ? 4 : 2;
  const size_t kpad = static_cast<size_t>((K + 63) / 64) * 64;
  const size_t Mpad = static_cast<size_t>((M + kBM - 1) / kBM) * kBM;
  uint8_t* a = static_cast<uint8_t*>(ws);
  uint8_t* b = a + ((ns * eb * kpad * Mpad + 1023) & ~size_t(1023));
  if (mode == 0) return launch_tc_mode<0>(M, N, K, L, ldl, U, ldu, C, ldc, st, track, a, b, s);
  return launch_tc_mode<1>(M, N, K, L, ldl, U, ldu, C, ldc, st, track, a, b, s);
}

}  // namespace prrp
