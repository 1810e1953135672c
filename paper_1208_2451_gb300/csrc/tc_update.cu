// Schur update A22 -= L21 A12 (Algorithm 1, line 7) on the tcgen05 tensor cores, for the
// mixed-precision forms: TF32 (one product) or a 3-term BF16 split (x = hi + mid + lo,
// six products hi*hi + hi*mid + mid*hi + hi*lo + lo*hi + mid*mid, about FP32 accuracy).
// Accumulation is FP32 in tensor memory; the FP64 trailing matrix is updated in the
// epilogue (C_ij -= acc_ij in FP64).  The same C -= L U form carries U12 and the final
// multipliers in those modes.  A second kernel further down computes the update to FP64
// accuracy from an exact fixed-point split into BF16 digits (the "FP64-accurate update").
//
// One persistent CTA per SM, warp-specialized, over 128 x 128 output tiles:
//   * warp 0 (one lane) streams every operand slice of a tile with TMA (K-major, 128-byte
//     swizzled rows, zero-padded to multiples of 128 rows and 64 k) into a ring of
//     shared-memory stages, each guarded by a full and an empty mbarrier;
//   * warp 1 (one lane) issues the tcgen05.mma instructions (M = 128, N = 128, 32 bytes of
//     k each) into one of two 128-column TMEM accumulators, commits each stage's MMAs to
//     its empty barrier and each finished tile to the accumulator's full barrier;
//   * warps 2..17 (four per TMEM lane quarter, each a 32 x 32 block of the tile) read the
//     other accumulator, release it, and update C in FP64.  Where C allows (16-byte
//     aligned, even leading dimension and width) the C boxes move HBM -> shared memory ->
//     HBM by TMA, loaded a tile ahead and updated in place in shared memory; otherwise each
//     block is transposed through shared memory and C is loaded and stored from registers
//     with row-contiguous, coalesced accesses.  Both track max |C| for the growth factor.
// So the HBM-bound epilogue of one tile overlaps the loads and MMAs of the next.  Every
// wait is bounded: on expiry the CTA records PRRP_ERR_TIMEOUT, frees its tensor memory
// and returns.
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

constexpr int kBM = 128, kBN = 128;
constexpr int kStage = 33;        // padded row of the 32 x 32 transpose stage (floats)
constexpr int kEpiWarps = 16;     // four warps per TMEM lane quarter, each a quarter of the columns
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kTmemCols = 2 * kBN;  // double-buffered accumulator
constexpr int kCSlots = 2;          // C boxes per epilogue warp and tile: 32 rows x 16 doubles
constexpr int kCBox = 32 * 128;     // bytes of one C box (128-byte rows, 128-byte swizzle)

// CT = 1: C moves through shared memory by TMA (needs a 16-byte aligned C, an even leading
// dimension and an even column count); CT = 0: the epilogue loads and stores C from
// registers.
template <int MODE, int CT>
struct TcCfg {
  static constexpr int EB = MODE == 0 ? 4 : 2;         // operand bytes per element
  static constexpr int CH = MODE == 0 ? 2 : 1;         // 128-byte chunks per 64-wide k block
  static constexpr int NS = MODE == 0 ? 1 : 3;         // slices per operand
  static constexpr int NP = MODE == 0 ? 1 : 6;         // slice products
  static constexpr int TILE_A = kBM * 128;             // bytes per slice-chunk
  static constexpr int TILE_B = kBN * 128;
  static constexpr int OPER_BYTES = NS * CH * (TILE_A + TILE_B);   // one pipeline stage
  static constexpr int EPI_BYTES = CT ? kEpiWarps * kCSlots * kCBox : kEpiWarps * 32 * kStage * 4;
  // as many operand stages as fit next to the epilogue buffers (static shared memory and
  // the 1 KB alignment slack kept aside)
  static constexpr int NSTAGE = (kSmemOptin - 512 - EPI_BYTES - 1024) / OPER_BYTES;
  static constexpr int SMEM = NSTAGE * OPER_BYTES + EPI_BYTES + 1024;
  static constexpr uint32_t IDESC = make_idesc(MODE == 0 ? 2u : 1u, kBM, kBN);
  static_assert(NSTAGE >= 1, "operand stages");
};

__constant__ int c_prod_a[6] = {0, 0, 1, 0, 2, 1};
__constant__ int c_prod_b[6] = {0, 1, 0, 2, 0, 1};

// float -> double with integer operations only: rebias the exponent and widen the
// mantissa.  Exact for normal values, inf and nan; zero and the FP32 subnormals (below
// 1.2e-38 in magnitude) become a signed zero.  On this GPU the FP64 pipe runs at 2
// operations per clock per SM, so the epilogue keeps it for the one operation that needs
// it, the subtraction (a hardware conversion here would be a second FP64-pipe op).
__device__ __forceinline__ double f2d_int(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xFFu;
  const uint32_t ee = (e == 0u) ? 0u : (e == 0xFFu ? 0x7FFu : e + 896u);
  const uint32_t mm = (e == 0u) ? 0u : (u & 0x7FFFFFu);
  const unsigned long long d = (static_cast<unsigned long long>(u & 0x80000000u) << 32) |
                               (static_cast<unsigned long long>(ee) << 52) |
                               (static_cast<unsigned long long>(mm) << 29);
  return __longlong_as_double(static_cast<long long>(d));
}

// Ask L2 to fetch the part of one row of C that a warp will update next: the 16-byte
// aligned interior of [p, p + ncols) (bulk prefetch wants 16-byte aligned address and size;
// the few bytes outside it are simply not prefetched).  Only addresses inside the row are
// named, so the hint never reaches past the matrix.
__device__ __forceinline__ void prefetch_row_l2(const double* p, int ncols) {
  if (ncols <= 0) return;
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(p);
  const uintptr_t lo = (a0 + 15) & ~uintptr_t(15);
  const uintptr_t hi = (a0 + static_cast<uintptr_t>(ncols) * 8u) & ~uintptr_t(15);
  if (hi > lo)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"(static_cast<uint32_t>(hi - lo))
                 : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* tm, const void* src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   reinterpret_cast<uint64_t>(tm)),
               "r"(x), "r"(y), "r"(smem_u32(src))
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// stores issued by this thread: wait until all but the newest N have read shared memory
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Persistent, warp-specialized: warp 0 (one lane) streams operand tiles with TMA into an
// NSTAGE ring, warp 1 (one lane) issues the MMAs into one of two TMEM accumulators, warps
// 2..9 drain the other accumulator into C.  Tiles are taken round-robin by CTA.
template <int MODE, int CT>
__global__ void __launch_bounds__(kThreads, 1) tc_update_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                const __grid_constant__ CUtensorMap tmB,
                                                                const __grid_constant__ CUtensorMap tmC,
                                                                int M, int N, int kblocks, int Mpad, int Npad,
                                                                double* __restrict__ C, long long ldc,
                                                                DevState* st, int track) {
  using Cfg = TcCfg<MODE, CT>;
  constexpr int NSTG = Cfg::NSTAGE;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[NSTG], empty[NSTG], accf[2], acce[2];
  __shared__ __align__(8) uint64_t cbar[CT ? kEpiWarps * kCSlots : 1];
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  if (dev_status(st) != 0) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tiles_n = Npad / kBN, tiles = (Mpad / kBM) * tiles_n;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int i = 0; i < NSTG; ++i) { mbar_init(&full[i], 1); mbar_init(&empty[i], 1); }
    for (int i = 0; i < 2; ++i) { mbar_init(&accf[i], 1); mbar_init(&acce[i], kEpiWarps); }
    if (CT)
      for (int i = 0; i < kEpiWarps * kCSlots; ++i) mbar_init(&cbar[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  unsigned long long cmax_bits = 0ull;          // max |C| as a non-negative IEEE bit pattern
  int p_it = 0;                                 // operand loads issued (producer lane)

  if (warp == 0) {
    if (lane == 0) {                                         // ---- TMA producer
      for (int tile = blockIdx.x; tile < tiles && !s_fail; tile += gridDim.x) {
        const int bm = (tile / tiles_n) * kBM, bn = (tile % tiles_n) * kBN;
        for (int kb = 0; kb < kblocks; ++kb, ++p_it) {
          const int s = p_it % NSTG;
          if (!mbar_wait_bounded(&empty[s], ((p_it / NSTG) & 1) ^ 1)) { s_fail = 1; break; }
          uint8_t* sA = base + s * Cfg::OPER_BYTES;
          uint8_t* sB = sA + Cfg::NS * Cfg::CH * Cfg::TILE_A;
          mbar_expect_tx(&full[s], Cfg::OPER_BYTES);
          for (int sl = 0; sl < Cfg::NS; ++sl)
            for (int c = 0; c < Cfg::CH; ++c) {
              const int x = kb * 64 + c * (128 / Cfg::EB);
              tma_load_2d(sA + (sl * Cfg::CH + c) * Cfg::TILE_A, &tmA, x, sl * Mpad + bm, &full[s]);
              tma_load_2d(sB + (sl * Cfg::CH + c) * Cfg::TILE_B, &tmB, x, sl * Npad + bn, &full[s]);
            }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {                                         // ---- MMA issuer
      int it = 0, tcount = 0;
      for (int tile = blockIdx.x; tile < tiles && !s_fail; tile += gridDim.x, ++tcount) {
        const int a = tcount & 1;
        if (!mbar_wait_bounded(&acce[a], ((tcount >> 1) & 1) ^ 1)) { s_fail = 1; break; }
        tc_fence_after();
        const uint32_t dt = tmem + a * kBN;
        for (int kb = 0; kb < kblocks; ++kb, ++it) {
          const int s = it % NSTG;
          if (!mbar_wait_bounded(&full[s], (it / NSTG) & 1)) { s_fail = 1; break; }
          tc_fence_after();
          uint8_t* sA = base + s * Cfg::OPER_BYTES;
          uint8_t* sB = sA + Cfg::NS * Cfg::CH * Cfg::TILE_A;
          for (int p = 0; p < Cfg::NP; ++p) {
            const int as = c_prod_a[p], bs = c_prod_b[p];
            for (int c = 0; c < Cfg::CH; ++c) {
              const uint64_t ad = sw128_desc(smem_u32(sA + (as * Cfg::CH + c) * Cfg::TILE_A));
              const uint64_t bd = sw128_desc(smem_u32(sB + (bs * Cfg::CH + c) * Cfg::TILE_B));
#pragma unroll
              for (int k = 0; k < 4; ++k)
                umma<MODE>(dt, ad + 2 * k, bd + 2 * k, Cfg::IDESC, (kb | p | c | k) != 0);
            }
          }
          umma_commit(&empty[s]);                            // frees the stage when done
        }
        if (s_fail) break;
        umma_commit(&accf[a]);                               // accumulator ready
      }
    }
  } else if constexpr (CT) {                                 // ---- epilogue warps, C by TMA
    // Warp (q, cq) owns rows 32q..32q+31 and columns 32cq..32cq+31 of every tile, as two
    // 32 x 16 boxes, one shared-memory slot each.  The boxes of the next tile are loaded
    // while the current tile drains: a slot is refilled as soon as the TMA store of its
    // previous contents has read it.  Lane i updates row i of a box in place.
    const int q = warp & 3, cq = (warp - 2) >> 2, ew = warp - 2;
    uint8_t* ring = base + NSTG * Cfg::OPER_BYTES + ew * kCSlots * kCBox;
    uint64_t* cb = &cbar[ew * kCSlots];
    uint32_t phase = 0u, pending = 0u;       // per-slot barrier parity; loads not yet consumed
    auto box_x = [&](int t, int slot) { return (t % tiles_n) * kBN + cq * 32 + slot * 16; };
    auto box_y = [&](int t) { return (t / tiles_n) * kBM + q * 32; };
    auto refill = [&](int t, int slot) {     // lane 0: load box `slot` of tile t if it holds C
      if (t < tiles && box_y(t) < M && box_x(t, slot) < N) {
        mbar_expect_tx(&cb[slot], kCBox);
        tma_load_2d(ring + slot * kCBox, &tmC, box_x(t, slot), box_y(t), &cb[slot]);
        pending |= 1u << slot;
      }
    };
    if (lane == 0)
      for (int slot = 0; slot < kCSlots; ++slot) refill(blockIdx.x, slot);
    int tcount = 0;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++tcount) {
      const int a = tcount & 1;
      // every lane observes the barrier itself; a timeout in any lane fails the whole warp
      if (!__all_sync(0xffffffffu, mbar_wait_bounded(&accf[a], (tcount >> 1) & 1))) { s_fail = 1; break; }
      tc_fence_after();
      uint32_t acc[32];
      tmem_ld32(tmem + a * kBN + (static_cast<uint32_t>(q * 32) << 16) + cq * 32, acc);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[a]);                  // accumulator free again
      const int y = box_y(tile), next = tile + gridDim.x;
      bool failed = false;
#pragma unroll
      for (int slot = 0; slot < kCSlots; ++slot) {
        const bool live = y < M && box_x(tile, slot) < N;
        if (live) {
          if (!__all_sync(0xffffffffu, mbar_wait_bounded(&cb[slot], (phase >> slot) & 1u))) { failed = true; break; }
          phase ^= 1u << slot;
          pending &= ~(1u << slot);
          uint8_t* row = ring + slot * kCBox + lane * 128;
#pragma unroll
          for (int p = 0; p < 8; ++p) {
            double2* cp = reinterpret_cast<double2*>(row + ((p ^ (lane & 7)) << 4));
            double2 cv = *cp;
            cv.x -= f2d_int(__uint_as_float(acc[slot * 16 + 2 * p]));
            cv.y -= f2d_int(__uint_as_float(acc[slot * 16 + 2 * p + 1]));
            *cp = cv;
            cmax_bits = max_bits(cmax_bits, max_bits(abs_bits(cv.x), abs_bits(cv.y)));
          }
          fence_proxy_async();                               // generic writes -> TMA store
          __syncwarp();
          if (lane == 0) tma_store_2d(&tmC, ring + slot * kCBox, box_x(tile, slot), y);
        }
        // the previous slot's store has read its box once at most the newest store is
        // pending: refill it with the next tile's box
        if (lane == 0 && slot > 0) {
          if (live) bulk_wait_read<1>(); else bulk_wait_read<0>();
          refill(next, slot - 1);
        }
        __syncwarp();
      }
      if (failed) { s_fail = 1; break; }
      if (lane == 0) {
        bulk_wait_read<0>();
        refill(next, kCSlots - 1);
      }
      __syncwarp();
    }
    if (lane == 0) {
      bulk_wait_all();                                       // stores finished
      for (int slot = 0; slot < kCSlots; ++slot)             // loads in flight after a failure
        if ((pending >> slot) & 1u) mbar_wait_bounded(&cb[slot], (phase >> slot) & 1u);
    }
    __syncwarp();
  } else {                                                   // ---- epilogue warps, C by registers
    const int q = warp & 3;                                  // TMEM lane quarter of this warp
    const int cq = (warp - 2) >> 2;                          // column quarter
    float* stage = reinterpret_cast<float*>(base + NSTG * Cfg::OPER_BYTES) + (warp - 2) * 32 * kStage;
    // each lane owns one row of this warp's 32 x 32 region of a tile: the row of the next
    // tile is prefetched into L2 while the current one drains
    auto prefetch_tile = [&](int t) {
      if (t >= tiles) return;
      const int r = (t / tiles_n) * kBM + q * 32 + lane, c = (t % tiles_n) * kBN + cq * 32;
      if (r < M && c < N) prefetch_row_l2(C + static_cast<long long>(r) * ldc + c, min(32, N - c));
    };
    prefetch_tile(blockIdx.x);
    int tcount = 0;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++tcount) {
      const int a = tcount & 1;
      const int bm = (tile / tiles_n) * kBM, bn = (tile % tiles_n) * kBN;
      prefetch_tile(tile + gridDim.x);
      if (!mbar_wait_bounded(&accf[a], (tcount >> 1) & 1)) { s_fail = 1; break; }
      tc_fence_after();
      const int rbase = bm + q * 32;
      const int nrows = min(32, M - rbase);
      {
        const int c0 = cq * 32;
        uint32_t r[32];
        tmem_ld32(tmem + a * kBN + (static_cast<uint32_t>(q * 32) << 16) + c0, r);
#pragma unroll
        for (int j = 0; j < 32; ++j) stage[lane * kStage + j] = __uint_as_float(r[j]);
        __syncwarp();
        const int col = bn + c0 + lane;
        if (col < N && nrows > 0) {
          double* cp = C + static_cast<long long>(rbase) * ldc + col;
          const int ldci = static_cast<int>(ldc);          // 32 rows x ldc fits in 32 bits
#pragma unroll
          for (int h16 = 0; h16 < 32; h16 += 16) {
            double cv[16];
#pragma unroll
            for (int rr = 0; rr < 16; ++rr)
              if (h16 + rr < nrows) cv[rr] = __ldcs(cp + (h16 + rr) * ldci);
#pragma unroll
            for (int rr = 0; rr < 16; ++rr)
              if (h16 + rr < nrows) {
                const double v = cv[rr] - f2d_int(stage[(h16 + rr) * kStage + lane]);
                __stcs(cp + (h16 + rr) * ldci, v);
                cmax_bits = max_bits(cmax_bits, abs_bits(v));
              }
          }
        }
        __syncwarp();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[a]);                  // accumulator free again
    }
  }
  if (track && warp >= 2) {
    for (int off = 16; off > 0; off >>= 1) {
      cmax_bits = max_bits(cmax_bits, __shfl_xor_sync(0xffffffffu, cmax_bits, off));
    }
    // NaN bit patterns sort above every finite value; the input scan rejects them earlier
    if (lane == 0) atomicMax(track == 2 ? &st->umax_bits : &st->gmax_bits, cmax_bits);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0 && lane == 0 && s_fail) {
    // operand loads still in flight after a failure: the last load into each stage
    for (int i = p_it - 1; i >= 0 && i >= p_it - NSTG; --i) mbar_wait_bounded(&full[i % NSTG], (i / NSTG) & 1);
  }
  if (s_fail && tid == 0) set_error(st, PRRP_ERR_TIMEOUT);
  __syncwarp();
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

// 2-D map over a [slices * rows_pad] x kpad row-major operand, box = 128 bytes x box_rows.
bool make_map(CUtensorMap* m, void* base, int mode, int rows_total, int kpad, int box_rows = 128) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const int eb = mode == 0 ? 4 : 2;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(kpad), static_cast<cuuint64_t>(rows_total)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(kpad) * eb};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(128 / eb), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, mode == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base,
                  dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// 2-D map over the FP64 matrix C (M x N, leading dimension ldc), box = 32 rows x 16
// doubles with 128-byte swizzle; rows and columns past the edge read as zero and are not
// written back.  Needs a 16-byte aligned C, an even ldc and an even N: the store clips the
// row at 16-byte granularity, so with an odd N it would also write column N.
bool make_c_map(CUtensorMap* m, double* C, int M, int N, long long ldc) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || (reinterpret_cast<uintptr_t>(C) & 15u) != 0 || (ldc & 1) != 0 || (N & 1) != 0) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(N), static_cast<cuuint64_t>(M)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ldc) * 8};
  cuuint32_t box[2] = {16, 32};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, C, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int MODE, int CT>
cudaError_t launch_tc_kernel(const CUtensorMap& ma, const CUtensorMap& mb, const CUtensorMap& mc, int M, int N,
                             int kblocks, int Mpad, int Npad, double* C, long long ldc, DevState* st, int track,
                             int max_ctas, cudaStream_t s) {
  using Cfg = TcCfg<MODE, CT>;
  cudaError_t e = smem_optin(tc_update_kernel<MODE, CT>);
  if (e != cudaSuccess) return e;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tiles = (Npad / kBN) * (Mpad / kBM);
  if (max_ctas > 0) sms = std::min(sms, max_ctas);
  tc_update_kernel<MODE, CT><<<std::min(tiles, sms), kThreads, Cfg::SMEM, s>>>(ma, mb, mc, M, N, kblocks, Mpad,
                                                                               Npad, C, ldc, st, track);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_tc_mode(int M, int N, int K, const double* L, long long ldl, const double* U, long long ldu,
                           double* C, long long ldc, DevState* st, int track, void* wsA, void* wsB,
                           int max_ctas, cudaStream_t s, cudaEvent_t after_split) {
  using Cfg = TcCfg<MODE, 0>;
  const int kblocks = (K + 63) / 64, kpad = kblocks * 64;
  const int Mpad = (M + kBM - 1) / kBM * kBM, Npad = (N + kBN - 1) / kBN * kBN;
  const long long ta = static_cast<long long>(Mpad) * kpad, tb = static_cast<long long>(Npad) * kpad;
  split_kernel<MODE, false><<<static_cast<int>(std::min<long long>((ta + 255) / 256, 152 * 16)), 256, 0, s>>>(
      L, ldl, M, K, Mpad, kpad, wsA);
  split_kernel<MODE, true><<<static_cast<int>(std::min<long long>((tb + 255) / 256, 152 * 16)), 256, 0, s>>>(
      U, ldu, N, K, Npad, kpad, wsB);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && after_split) e = cudaEventRecord(after_split, s);
  if (e != cudaSuccess) return e;
  CUtensorMap ma, mb, mc;
  if (!make_map(&ma, wsA, MODE, Cfg::NS * Mpad, kpad) || !make_map(&mb, wsB, MODE, Cfg::NS * Npad, kpad))
    return cudaErrorInvalidValue;
  if (make_c_map(&mc, C, M, N, ldc))
    return launch_tc_kernel<MODE, 1>(ma, mb, mc, M, N, kblocks, Mpad, Npad, C, ldc, st, track, max_ctas, s);
  return launch_tc_kernel<MODE, 0>(ma, mb, ma, M, N, kblocks, Mpad, Npad, C, ldc, st, track, max_ctas, s);
}


// ---------------------------------------------------------------- FP64-accurate update
//
// C -= L U to FP64 accuracy on the BF16 tensor cores by an exact fixed-point split (the
// Ozaki scheme).  Row r of L is scaled by 2^-e_r, e_r the least power of two above the
// row's max |l|, and cut into kOzS signed base-128 digits:
//     l_rk = 2^e_r sum_p L_p[r, k] 128^-(p+1),   |L_0| <= 128,  |L_p| <= 64 (p >= 1),
// leaving under 2^-57 of the row's scale; columns of U likewise with 2^f_c.  Digits are
// integers of at most 8 significant bits, so for K <= 64 every BF16 product L_p U_q is an
// integer below 2^20 that FP32 accumulation holds exactly, and the products of one
// diagonal d = p + q share a TMEM accumulator (below 2^22, still exact).  The diagonals
// d <= kOzS - 1 (36 products) are kept; the dropped ones and the digits' remainders are
// below 2^-53 sum_k |l_rk| |u_kc| in practice.  The epilogue assembles
//     T = sum_d acc_d 2^(7 (7 - d) - 8)    (|T| < 2^62)
// in 64-bit integers, exactly for d <= 5 and with the last two diagonals shifted down by
// 1 and 8 bits (floor: under 2 units of T, i.e. 2^(e_r + f_c - 54)), and applies it with
// the scale 2^(e_r + f_c - 55): one conversion and one FMA on the FP64 pipe per element
// of C, against 2K for the plain product.
constexpr int kOzS = 8;                   // digits per operand
constexpr int kOzBN = 64;                 // tile columns: kOzS accumulators x 64 = 512 TMEM columns
constexpr int kOzEpi = 8;                 // epilogue warps: 4 TMEM lane quarters x 2 column halves
constexpr int kOzThreads = 64 + 32 * kOzEpi;
constexpr int kOzTileA = kBM * 128;       // one digit slice of L: 128 rows x 64 BF16
constexpr int kOzTileB = kOzBN * 128;     // one digit slice of U: 64 rows x 64 BF16
constexpr int kOzStage = kOzS * (kOzTileA + kOzTileB);   // every slice of a tile: 192 KB
constexpr int kOzXP = 9;                  // padded row (doubles) of an epilogue warp's 32 x 8 stage
constexpr int kOzSmem = kOzStage + kOzEpi * 32 * kOzXP * 8 + 1024;
static_assert(kOzSmem + 512 <= kSmemOptin, "one operand stage");
constexpr uint32_t kOzIdesc = make_idesc(1u, kBM, kOzBN);

// An accumulator's integer a (|a| < 2^22) as the bits of a + 1.5 2^23: a + kOzBias.
constexpr unsigned kOzBias = 0x4B400000u;
__device__ __forceinline__ uint32_t oz_bits(uint32_t acc) {
  return __float_as_uint(__uint_as_float(acc) + 12582912.0f);
}
// The biases' total under the epilogue's weights, modulo 2^64 (unsigned arithmetic wraps).
constexpr unsigned long long kOzBiasSum =
    static_cast<unsigned long long>(kOzBias) * ((1ull << 41) + (1ull << 34) + (1ull << 27) + (1ull << 20) +
                                                (1ull << 13) + (1ull << 6)) +
    kOzBias / 2 + kOzBias / 256;
static_assert(kOzBias % 256 == 0, "the floors pass through the bias");

// 2^k as a double: subnormal down to 2^-1074, 0 below (an underflowing product is dropped),
// 2^1023 above the range.
__device__ __forceinline__ double pow2i(int k) {
  if (k < -1074) return 0.0;
  if (k < -1022) return __longlong_as_double(1ll << (k + 1074));
  if (k > 1023) k = 1023;
  return __longlong_as_double(static_cast<long long>(k + 1023) << 52);
}

// BF16 bits of an integer-valued double with |d| <= 256 (at most 8 significant bits, so
// the truncated mantissa is exact), by integer operations.
__device__ __forceinline__ unsigned short d2bf16_int(double d) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(d));
  if ((u << 1) == 0ull) return 0;
  const unsigned sign = static_cast<unsigned>(u >> 63);
  const unsigned e = static_cast<unsigned>((u >> 52) & 0x7FFu) - 1023u + 127u;
  const unsigned mant = static_cast<unsigned>((u >> 45) & 0x7Fu);
  return static_cast<unsigned short>((sign << 15) | (e << 7) | mant);
}

// Digits of the operand lines: line r (a row of L, or with COLS a column of U) of K <= 64
// entries, one warp per line.  dst[p][r][k] (rows_pad x 64 BF16 per slice); exps[r] = e_r.
template <bool COLS>
__global__ void ozaki_split_kernel(const double* __restrict__ src, long long ld, int rows, int K, int rows_pad,
                                   unsigned short* __restrict__ dst, int* __restrict__ exps) {
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (int r = blockIdx.x * wpb + (threadIdx.x >> 5); r < rows_pad; r += gridDim.x * wpb) {
    double x[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = lane + 32 * h;
      x[h] = (r < rows && k < K) ? (COLS ? src[static_cast<long long>(k) * ld + r] : src[static_cast<long long>(r) * ld + k])
                                 : 0.0;
    }
    unsigned long long m = max_bits(abs_bits(x[0]), abs_bits(x[1]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = max_bits(m, __shfl_xor_sync(0xffffffffu, m, off));
    // max |x| < 2^e (the scale 2^-e is exact, subnormal for e = 1023); a line whose max
    // is 2^1023 or more is scaled by 2^-1023 only, its leading digits reach 256 and the
    // exactness bounds no longer hold: such entries are outside this mode's range
    int e = m == 0ull ? 0 : static_cast<int>((m >> 52) & 0x7FFu) - 1022;
    e = min(max(e, -1021), 1023);
    if (lane == 0 && r < rows) exps[r] = e;
    const double sc = pow2i(-e);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      double y = x[h] * sc;                     // exact; |y| < 1
      unsigned short* out = dst + static_cast<long long>(r) * 64 + lane + 32 * h;
#pragma unroll
      for (int p = 0; p < kOzS; ++p) {
        y *= 128.0;                             // exact
        const double d = rint(y);
        y -= d;                                 // exact
        out[static_cast<long long>(p) * rows_pad * 64] = d2bf16_int(d);
      }
    }
  }
}

// Persistent, warp-specialized, one 128 x 64 tile at a time: warp 0 (one lane) loads every
// digit slice of the tile with TMA into the one operand stage; warp 1 (one lane) issues the
// 36 slice products (4 MMAs of K = 16 each) into the 8 diagonal accumulators; warps 2..9
// assemble and apply them.  The next tile's operands load while the epilogue drains.
__global__ void __launch_bounds__(kOzThreads, 1) ozaki_update_kernel(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N, int Mpad,
    int Npad, const int* __restrict__ rexp, const int* __restrict__ cexp, double* __restrict__ C, long long ldc,
    DevState* st, int track) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full, empty, accf, acce;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  if (dev_status(st) != 0) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = base;
  uint8_t* sB = base + kOzS * kOzTileA;
  const int tiles_n = Npad / kOzBN, tiles = (Mpad / kBM) * tiles_n;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(kOzS * kOzBN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    mbar_init(&full, 1);
    mbar_init(&empty, 1);
    mbar_init(&accf, 1);
    mbar_init(&acce, kOzEpi);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  unsigned long long cmax_bits = 0ull;
  int p_it = 0;                                  // tiles whose operands were requested

  if (warp == 0) {
    if (lane == 0) {                                         // ---- TMA producer
      for (int tile = blockIdx.x; tile < tiles && !s_fail; tile += gridDim.x, ++p_it) {
        const int bm = (tile / tiles_n) * kBM, bn = (tile % tiles_n) * kOzBN;
        if (!mbar_wait_bounded(&empty, (p_it & 1) ^ 1)) { s_fail = 1; break; }
        mbar_expect_tx(&full, kOzStage);
        for (int sl = 0; sl < kOzS; ++sl) {
          tma_load_2d(sA + sl * kOzTileA, &tmA, 0, sl * Mpad + bm, &full);
          tma_load_2d(sB + sl * kOzTileB, &tmB, 0, sl * Npad + bn, &full);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {                                         // ---- MMA issuer
      int it = 0;
      for (int tile = blockIdx.x; tile < tiles && !s_fail; tile += gridDim.x, ++it) {
        if (!mbar_wait_bounded(&acce, (it & 1) ^ 1)) { s_fail = 1; break; }
        if (!mbar_wait_bounded(&full, it & 1)) { s_fail = 1; break; }
        tc_fence_after();
        for (int p = 0; p < kOzS; ++p) {
          const uint64_t ad = sw128_desc(smem_u32(sA + p * kOzTileA));
          for (int q = 0; p + q < kOzS; ++q) {
            const uint64_t bd = sw128_desc(smem_u32(sB + q * kOzTileB));
            const uint32_t dt = tmem + static_cast<uint32_t>((p + q) * kOzBN);
            // p = 0 opens diagonal q; later p add to it
#pragma unroll
            for (int k = 0; k < 4; ++k) umma<1>(dt, ad + 2 * k, bd + 2 * k, kOzIdesc, (p | k) != 0);
          }
        }
        umma_commit(&empty);                                 // operand stage free
        umma_commit(&accf);                                  // accumulators ready
      }
    }
  } else {                                                   // ---- epilogue warps
    // a warp reads TMEM lanes 32 (warp % 4) .. + 31: warps 2..9 cover each lane quarter
    // twice, once per 32-column half of the tile
    const int q = warp & 3, h = (warp - 2) >> 2;
    int tcount = 0;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++tcount) {
      const int bm = (tile / tiles_n) * kBM, bn = (tile % tiles_n) * kOzBN;
      if (!__all_sync(0xffffffffu, mbar_wait_bounded(&accf, tcount & 1))) { s_fail = 1; break; }
      tc_fence_after();
      const uint32_t tb = tmem + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(h * 32);
      // T = sum_{d <= 5} a_d 2^(41 - 7 d) + floor(a_6 / 2) + floor(a_7 / 256), a_d the integer
      // in accumulator d.  Each a_d is read as the bits b_d = a_d + kOzBias of a_d + 1.5 2^23
      // (one FP32 add); the b_d are summed with their weights modulo 2^64 by wide integer
      // multiply-adds (kOzBias is a multiple of 256, so the floors pass through it), and the
      // biases' weighted total comes off once.  |T| < 2^62, so the wrapped sum is T exactly.
      unsigned long long T[32];
      uint32_t r[32];
      tmem_ld32(tb, r);                                      // diagonal 0: 2^41
#pragma unroll
      for (int j = 0; j < 32; ++j) T[j] = static_cast<unsigned long long>(oz_bits(r[j]) << 9) << 32;
      tmem_ld32(tb + static_cast<uint32_t>(kOzBN), r);       // diagonal 1: 2^34
#pragma unroll
      for (int j = 0; j < 32; ++j) T[j] += static_cast<unsigned long long>(oz_bits(r[j]) << 2) << 32;
#pragma unroll 1
      for (int d = 2; d < kOzS - 2; ++d) {                   // diagonals 2..5: 2^27 .. 2^6
        tmem_ld32(tb + static_cast<uint32_t>(d * kOzBN), r);
        const uint32_t wgt = 1u << (41 - 7 * d);
#pragma unroll
        for (int j = 0; j < 32; ++j) T[j] += static_cast<unsigned long long>(oz_bits(r[j])) * wgt;
      }
      tmem_ld32(tb + static_cast<uint32_t>((kOzS - 2) * kOzBN), r);   // diagonal 6: 2^-1
#pragma unroll
      for (int j = 0; j < 32; ++j) T[j] += oz_bits(r[j]) >> 1;
      tmem_ld32(tb + static_cast<uint32_t>((kOzS - 1) * kOzBN), r);   // diagonal 7: 2^-8
#pragma unroll
      for (int j = 0; j < 32; ++j) T[j] = T[j] + (oz_bits(r[j]) >> 8) - kOzBiasSum;
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce);                     // accumulators free again
      // lane = row of the 32 x 32 block; C is updated through a 32 x 8 shared-memory stage
      // per chunk of columns, so that a warp's load or store touches 4 rows x 8 columns
      // (4 x 64 contiguous bytes) rather than 32 rows
      const int row0 = bm + q * 32, c0 = bn + h * 32;
      const int nrows = min(32, M - row0), ncols = min(32, N - c0);
      if (nrows > 0 && ncols > 0) {
        double* stg = reinterpret_cast<double*>(base + kOzStage) + (warp - 2) * 32 * kOzXP;
        const int cl = lane & 7, rl = lane >> 3;          // this lane: column cl, rows rl + 4 i
        int er[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) er[i] = rl + 4 * i < nrows ? __ldg(rexp + row0 + rl + 4 * i) - 55 : 0;
#pragma unroll
        for (int j0 = 0; j0 < 32; j0 += 8) {
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) stg[lane * kOzXP + jj] = static_cast<double>(static_cast<long long>(T[j0 + jj]));
          __syncwarp();
          const int col = c0 + j0 + cl;
          if (j0 + cl < ncols) {
            const int ec = __ldg(cexp + col);
            double cv[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
              if (rl + 4 * i < nrows) cv[i] = __ldcs(C + static_cast<long long>(row0 + rl + 4 * i) * ldc + col);
#pragma unroll
            for (int i = 0; i < 8; ++i)
              if (rl + 4 * i < nrows) {
                const int r = rl + 4 * i;
                const double v = fma(-stg[r * kOzXP + cl], pow2i(er[i] + ec), cv[i]);
                __stcs(C + static_cast<long long>(row0 + r) * ldc + col, v);
                cmax_bits = max_bits(cmax_bits, abs_bits(v));
              }
          }
          __syncwarp();
        }
      }
    }
  }
  if (track && warp >= 2) {
    for (int off = 16; off > 0; off >>= 1) cmax_bits = max_bits(cmax_bits, __shfl_xor_sync(0xffffffffu, cmax_bits, off));
    if (lane == 0) atomicMax(track == 2 ? &st->umax_bits : &st->gmax_bits, cmax_bits);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0 && lane == 0 && s_fail && p_it > 0) mbar_wait_bounded(&full, (p_it - 1) & 1);   // loads in flight
  if (s_fail && tid == 0) set_error(st, PRRP_ERR_TIMEOUT);
  __syncwarp();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kOzS * kOzBN) : "memory");
}

size_t ozaki_ws_bytes(int M, int N) {
  const size_t Mpad = static_cast<size_t>((M + kBM - 1) / kBM) * kBM;
  const size_t Npad = static_cast<size_t>((N + kOzBN - 1) / kOzBN) * kOzBN;
  return kOzS * 128 * (Mpad + Npad) + 4 * (Mpad + Npad) + 2048;
}

cudaError_t launch_ozaki(int M, int N, int K, const double* L, long long ldl, const double* U, long long ldu,
                         double* C, long long ldc, DevState* st, int track, void* ws, int max_ctas,
                         cudaStream_t s) {
  if (K > 64) return cudaErrorInvalidValue;
  const int Mpad = (M + kBM - 1) / kBM * kBM, Npad = (N + kOzBN - 1) / kOzBN * kOzBN;
  uint8_t* w = static_cast<uint8_t*>(ws);
  unsigned short* da = reinterpret_cast<unsigned short*>(w);
  unsigned short* db = reinterpret_cast<unsigned short*>(w + static_cast<size_t>(kOzS) * 128 * Mpad);
  int* rexp = reinterpret_cast<int*>(w + static_cast<size_t>(kOzS) * 128 * (Mpad + Npad));
  int* cexp = rexp + Mpad;
  ozaki_split_kernel<false><<<std::min((Mpad + 7) / 8, 152 * 8), 256, 0, s>>>(L, ldl, M, K, Mpad, da, rexp);
  ozaki_split_kernel<true><<<std::min((Npad + 7) / 8, 152 * 8), 256, 0, s>>>(U, ldu, N, K, Npad, db, cexp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  CUtensorMap ma, mb;
  if (!make_map(&ma, da, 1, kOzS * Mpad, 64, kBM) || !make_map(&mb, db, 1, kOzS * Npad, 64, kOzBN))
    return cudaErrorInvalidValue;
  if ((e = smem_optin(ozaki_update_kernel)) != cudaSuccess) return e;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tiles = (Mpad / kBM) * (Npad / kOzBN);
  if (max_ctas > 0) sms = std::min(sms, max_ctas);
  ozaki_update_kernel<<<std::min(tiles, sms), kOzThreads, kOzSmem, s>>>(ma, mb, M, N, Mpad, Npad, rexp, cexp, C,
                                                                         ldc, st, track);
  return cudaGetLastError();
}
}  // namespace

size_t tc_workspace_bytes(int prec, int M, int N, int K) {
  if (prec == PRRP_FP64_EMU) return ozaki_ws_bytes(M, N);
  const int mode = prec == PRRP_TF32 ? 0 : 1;
  const int ns = mode == 0 ? 1 : 3, eb = mode == 0 ? 4 : 2;
  const size_t kpad = static_cast<size_t>((K + 63) / 64) * 64;
  const size_t Mpad = static_cast<size_t>((M + kBM - 1) / kBM) * kBM;
  const size_t Npad = static_cast<size_t>((N + kBN - 1) / kBN) * kBN;
  return ns * eb * kpad * (Mpad + Npad) + 2048;
}

cudaError_t launch_tc_update(int prec, int M, int N, int K, const double* L, long long ldl, const double* U,
                             long long ldu, double* C, long long ldc, DevState* st, int track, void* ws,
                             cudaStream_t s, int max_ctas, cudaEvent_t after_split) {
  if (M <= 0 || N <= 0 || K <= 0) return after_split ? cudaEventRecord(after_split, s) : cudaSuccess;
  if (prec == PRRP_FP64_EMU) {
    cudaError_t e = launch_ozaki(M, N, K, L, ldl, U, ldu, C, ldc, st, track, ws, max_ctas, s);
    return (e == cudaSuccess && after_split) ? cudaEventRecord(after_split, s) : e;
  }
  const int mode = prec == PRRP_TF32 ? 0 : 1;
  const int ns = mode == 0 ? 1 : 3, eb = mode == 0 ? 4 : 2;
  const size_t kpad = static_cast<size_t>((K + 63) / 64) * 64;
  const size_t Mpad = static_cast<size_t>((M + kBM - 1) / kBM) * kBM;
  uint8_t* a = static_cast<uint8_t*>(ws);
  uint8_t* b = a + ((ns * eb * kpad * Mpad + 1023) & ~size_t(1023));
  if (mode == 0) return launch_tc_mode<0>(M, N, K, L, ldl, U, ldu, C, ldc, st, track, a, b, max_ctas, s, after_split);
  return launch_tc_mode<1>(M, N, K, L, ldl, U, ldu, C, ldc, st, track, a, b, max_ctas, s, after_split);
}

}  // namespace prrp
