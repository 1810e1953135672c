// Host-side launchers of the LU_PRRP kernels (internal to libprrp.so).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "common.cuh"

namespace prrp {

constexpr int kXVal = 3;   // doubles per interchange exchange record (the value; 2 spare)
constexpr int kQStride = kMaxW + 2;   // doubles per QRCP record: the row, then alpha and beta
constexpr int kQKeyStride = 1;        // u64 per QRCP key: a step's keys are contiguous
// QRCP key and record arrays rotate over kQSlots steps; the exchange fences once every
// kQFenceEvery steps, and kQSlots >= 2 kQFenceEvery + 2 keeps two fences between a slot's
// preparation and its next use
constexpr int kQFenceEvery = 4;
constexpr int kQSlots = 2 * kQFenceEvery + 2;
static_assert(kQSlots >= 2 * kQFenceEvery + 2 && kQFenceEvery >= 1,
              "a slot's preparation must be released and acquired before its reuse");
constexpr unsigned char kQSentinelByte = 0xFF;   // fills every record slot at launch
// SM split of the tensor-core modes (prrp_ctx_set_sm_split): panel CTAs, block-stream CTAs
constexpr int kSplitPanelDefault = 64;
// TF32 / 3xBF16 at n <= kSplitSmallN: the panels' share of the work is larger, and 96
// panel CTAs were faster (n = 8192, 3xBF16: 51.8 against 55.2 ms; n = 16384: 64 best)
constexpr int kSplitPanelSmallN = 96;
constexpr int kSplitSmallN = 10240;
constexpr int kSplitBlkDefault = 8;

struct PanelParams {
  const double* P;        // m x w panel, row-major
  long long ldp;
  int m, w;
  double tau;
  int max_swaps;
  int col_offset;         // global column of the panel's first column (for info)
  double* L21;            // (m - w) x w output, row-major
  int ldl;
  int* order;             // m ints (final position -> panel row) or nullptr
  int* pairs;             // (dst, src) row moves, 2 ints each, or nullptr
  DevState* st;
  double* xval;           // interchange exchange records: [2][G][kXVal] (value)
  int2* xkey;             // [2][G] (tie-breaks)
  double* xvec;           // [2][G][kMaxW] (row)
  unsigned long long* qkey;   // QRCP step keys [kQSlots][G][kQKeyStride], zero at launch
  double* qrow;               // QRCP records [kQSlots][G][kQStride], kQSentinelByte at launch
  int rows_per_cta;
  int cluster_rows;       // panels of at most this many rows run as one cluster (0: default)
  int nopivot;            // 1: unpivoted QR of the panel (CALU_PRRP's L21), no interchanges
};

int panel_width_class(int w);
size_t panel_smem_for(int w, int rows_per_cta);
cudaError_t launch_panel(const PanelParams& p, int G, cudaStream_t stream);
// A cooperative launch that waits, through a per-device event chain, for the previous
// cooperative launch of the library on any stream (two partially resident cooperative
// grids could otherwise wait on each other).
cudaError_t launch_cooperative_chained(const void* func, int grid, int threads, void** args, size_t smem,
                                       cudaStream_t stream);

// Trees of strong RRQRs over a panel's rows, one CTA per node (calu.cu), on the m x w
// panel P (row-major, ldp) whose first row is row k0 of A:
//   mode 0 (CALU_PRRP, Section 3.1): leaves of `leaf` rows (the last takes the remainder),
//     a binary tree; levels [level0, level1) in one launch with grid barriers between them;
//   mode 1 (block parallel LU_PRRP, Section 5): nleaf blocks of `leaf` rows (the last takes
//     the remainder), the same binary tree; mode 2 (block pairwise): a flat tree, level i
//     merges positions 0..w-1 with block i.  In modes 1 and 2 one launch runs one level
//     (level0 + 1 == level1), and each node also writes D = (R11^-1 R12)^T of the rows it
//     eliminates into their panel columns (Pw) and tracks max |D| in st->l21_bits.
// pmap (m ints, identity before level 0) maps position -> panel row; a node's selected
// rows take its first w positions.  w <= 64; every node holds at most 255 rows.
// Interchanges are added to st->swaps_total.
struct TournParams {
  const double* P;
  double* Pw;
  long long ldp;
  int m, w, leaf, nleaf, height;
  int mode, level0, level1;
  double tau;
  int max_swaps;
  int col_offset;
  int* pmap;
  DevState* st;
};
constexpr int kTreeNodeMaxRows = 255;
cudaError_t launch_tournament(const TournParams& p, int num_sms, cudaStream_t s);
// Modes 1 and 2, after the level's node launch: every row the level's nodes eliminated
// gets A_e(k0+w:n) -= D_e A_sel(k0+w:n) (the node's selected rows, not yet updated in this
// panel); max |A_e| into st->gmax_bits.  A is the whole matrix, row-major.
cudaError_t launch_tree_eliminate(const TournParams& p, double* A, long long lda, int n, int k0,
                                  int num_sms, cudaStream_t s);
// Rows k0 + i (all n columns) and perm[k0 + i] take those at k0 + pmap[i], i < m, through
// tmp (m x n doubles) and ptmp (m ints); rows with pmap[i] == i are not touched.
cudaError_t launch_gather_permute(double* A, long long lda, int n, int k0, int m, const int* pmap, int* perm,
                                  double* tmp, int* ptmp, DevState* st, cudaStream_t s);

// max |a_ij| and non-finite detection over an n x n row-major matrix.
cudaError_t launch_scan(const double* A, long long lda, int n, DevState* st, cudaStream_t s);

// Row moves for rows k0.. of A (all n columns) and perm: A[k0+dst] = A_old[k0+src].
cudaError_t launch_permute(double* A, long long lda, int n, int k0, const int* pairs,
                           int max_pairs, int* perm, DevState* st, cudaStream_t s);

// C -= L * U in FP64 (DFMA), C m x n, L m x k, U k x n, k <= kMaxW; tracks max |C| into
// st->gmax_bits when track != 0.  one_per_sm: 64 x 64 tiles, one persistent CTA per SM,
// tiles claimed from the device counter tile_ctr when it is given (zeroed on stream s
// before the launch; one counter per concurrently running update).
cudaError_t launch_gemm_fp64(int m, int n, int k, const double* L, long long ldl,
                             const double* U, long long ldu, double* C, long long ldc,
                             DevState* st, int track, int num_sms, cudaStream_t s, int one_per_sm = 0,
                             unsigned* tile_ctr = nullptr);

// Same update on tcgen05 tensor cores, prec = PRRP_TF32 or PRRP_BF16X3 (FP32 accumulation,
// FP64 C) or PRRP_FP64_EMU (exact digit split); ws holds the split operands
// (tc_workspace_bytes).  Both operands are split into ws before C is touched, so C may
// alias L or U.  track: 0 none, 1 max |C| into st->gmax_bits, 2 into st->umax_bits.
// max_ctas > 0 caps the persistent grid (one CTA per SM), leaving the other SMs free for
// kernels that run beside it.
size_t tc_workspace_bytes(int prec, int m, int n, int k);
// after_split, when given, is recorded on s once both operands are in ws: from then on
// L and U may change.
cudaError_t launch_tc_update(int prec, int m, int n, int k, const double* L, long long ldl,
                             const double* U, long long ldu, double* C, long long ldc, DevState* st,
                             int track, void* ws, cudaStream_t s, int max_ctas = 0,
                             cudaEvent_t after_split = nullptr);

// Aggregated update of the mixed-precision forms (one rank-NB product per block of panels).
// Block width limit: with TF32 operands, wider blocks no longer precondition FP64
// refinement at kappa = 1e4 (the rank-NB product takes the block's U rows, not the
// unreduced A12 of the per-panel form).
constexpr int kAggMaxNB = 256;
// Rows that moved between the block's start (perm0: row ids at positions K0..K0+rows-1)
// and now (perm): (i, src) position pairs relative to K0 into pairs, their number into
// *count (at most cap); pos0 is n ints of scratch.
cudaError_t launch_block_pairs(const int* perm0, const int* perm, int K0, int rows, int* pos0, int* pairs,
                               int* count, int cap, DevState* st, cudaStream_t s);
// The moves of those pairs over columns c0..c0+nc-1, through tmp (cap x nc doubles).
cudaError_t launch_block_moves(double* A, long long lda, int K0, int c0, int nc, const int* pairs,
                               const int* count, int cap, double* tmp, DevState* st, cudaStream_t s);

// GEPP on the w x w diagonal block at A[k0][k0]; in-block pivots to ipiv, perm updated,
// max |U11| tracked.
cudaError_t launch_diag_gepp(double* A, long long lda, int k0, int w, int* ipiv, int* perm,
                             DevState* st, cudaStream_t s);

// Block rows k0..k0+w-1: apply ipiv to columns [0, k0) and [k0+w, n); U12 = L11^-1 A12.
// solve = 0: only GEPP's interchanges, on every column outside the block (the triangular
// solve then runs elsewhere).
cudaError_t launch_u12(double* A, long long lda, int n, int k0, int w, const int* ipiv,
                       DevState* st, cudaStream_t s, int solve = 1);
// E = [I - L11^-1 ; I - L11] (2 w x w, ld w) for the tensor-core form of U12 and of the
// final multipliers (low-precision modes; L11^-1 formed in FP32).
cudaError_t launch_tri_blocks(const double* A, long long lda, int k0, int w, double* E, DevState* st,
                              cudaStream_t s);
// A[k0 + w + r][k0 + c] = L21[r][src(c)]: the multipliers with GEPP's column interchanges.
cudaError_t launch_lfix_copy(double* A, long long lda, int n, int k0, int w, const double* L21, int ldl21,
                             const int* ipiv, DevState* st, cudaStream_t s);

// Rows k0+w..n-1: A[r][k0:k0+w] = (L21buf[r] with columns interchanged by ipiv) * L11.
cudaError_t launch_lfix(double* A, long long lda, int n, int k0, int w, const double* L21,
                        int ldl21, const int* ipiv, DevState* st, cudaStream_t s);

cudaError_t launch_iota(int* p, int n, cudaStream_t s);
cudaError_t launch_wait_selftest(DevState* st, cudaStream_t s);

// Batched small systems (batch.cu): one CTA per system, persistent over a work list.
struct BatchLaunch {
  int count;
  const int* order;
  const int* n;
  const double* const* A;
  const int* lda;
  const int* nrhs;
  double* const* B;
  const int* ldb;
  int* const* perm_out;
  int b;
  double tau;
  int max_swaps;
  int refine_max_iter;
  double refine_target;
  int nmax;
  void* wsW;
  void* wsT;
  int tmp_rows;
  double* wsV;
  int* wsI;
  int* status;
  int* iters;
  double* eta0;
  double* eta;
  unsigned* counter;
};
size_t batch_smem_bytes(int nmax, int b);
int batch_max_width();
cudaError_t prepare_batch(int nmax, int b);
// rb: rows of L21 per warp pass in the Schur update (1 or 2; FP64 always 1), picked by
// the autotuner
cudaError_t launch_batch(int fp64, int grid, int rb, const BatchLaunch& L, cudaStream_t s);
cudaError_t launch_batch_fill(double* A, int n, int count, double* B, cudaStream_t s);

// Solve kernels (solve.cu).
cudaError_t launch_norm1(const double* A, long long lda, int n, double* out, cudaStream_t s);
cudaError_t launch_gather_rows(const double* B, long long ldb, const int* perm, int n, int nrhs,
                               double* Y, cudaStream_t s);
// Inverses of the 64 x 64 diagonal blocks of L (unit lower) and U, as T = float (fp32) or
// double: Dinv[2][nb][64 x 64] row-major, L first.
cudaError_t launch_invert_diag(const double* LU, long long lda, int n, void* dinv, int fp32, cudaStream_t s);
// Y <- L^-1 Y (lower) or U^-1 Y with the factors LU (T, leading dimension lda) and their
// inverted diagonal blocks; Y is n x nrhs row-major (T); counters: nb unsigned scratch.
cudaError_t launch_trsv(const void* LU, long long lda, const void* dinv, int n, void* Y, int nrhs, int lower,
                        int fp32, unsigned* counters, cudaStream_t s);
// Out <- L^-1 In (lower) or U^-1 In in one launch, for 1 <= nrhs <= kChainRhs.  In is
// overwritten (scratch); In and Out distinct, n x nrhs row-major (T).  counters:
// trsv_counter_words(n) unsigned; word 0 must be 0 on entry and is left holding the site
// of a wait that ran out (checked and cleared by the host), the rest is reset here.
constexpr int kChainRhs = 16;
constexpr int kTrsvCounterHead = 64;   // words before the per-block counters
inline size_t trsv_counter_words(int n) { return kTrsvCounterHead + 2 * (size_t)((n + 63) / 64); }
// One CTA of the FP32 substitution holding the ticket of block 1 of a two-block system whose
// block 0 nobody solves: its wait runs out.  scratch: kChainSelftestFloats floats.
constexpr size_t kChainSelftestFloats = 128 * 128 + 2 * 2 * 4096 + 2 * 128;
cudaError_t launch_trsv_chain_selftest(float* scratch, unsigned* counters, const DevState* st, cudaStream_t s);
cudaError_t launch_trsv_chain(const void* LU, long long lda, const void* dinv, int n, void* In, void* Out,
                              int nrhs, int lower, int fp32, unsigned* counters, const DevState* st,
                              cudaStream_t s);
cudaError_t launch_convert_lu32(const double* LU, long long lda, int n, float* out, cudaStream_t s);
cudaError_t launch_gather_rows32(const double* B, long long ldb, const int* perm, int n, int nrhs, float* Y,
                                 cudaStream_t s);
cudaError_t launch_axpy_rows32(double* X, long long ldx, const float* D, double alpha, int n, int nrhs,
                               cudaStream_t s);
// GMRES-based refinement (blocks of nrhs independent columns, n x nrhs row-major):
// Y = A X; out[i][c] = <V_i(:,c), W(:,c)> for i < nvec; W += sign * sum_i coef[i][c] V_i;
// Y = scale[c] * X (X FP64, or FP32 when x32 is given; scale may be null).
cudaError_t launch_matvec(const double* A, long long lda, int n, const double* X, long long ldx, int nrhs,
                          double* Y, cudaStream_t s);
cudaError_t launch_block_dots(const double* V, int nvec, int n, int nrhs, const double* W, double* out,
                              cudaStream_t s);
cudaError_t launch_block_axpy(const double* V, int nvec, int n, int nrhs, const double* coef, double sign,
                              double* W, cudaStream_t s);
cudaError_t launch_scale_cols(const double* X, const float* x32, int n, int nrhs, const double* scale, double* Y,
                              cudaStream_t s);
cudaError_t launch_residual(const double* A, long long lda, int n, const double* X, long long ldx,
                            int nrhs, const double* B, long long ldb, double* R, double* norms,
                            cudaStream_t s);
cudaError_t launch_axpy_rows(double* X, long long ldx, const double* D, double alpha, int n,
                             int nrhs, cudaStream_t s);
cudaError_t launch_copy_rows(const double* src, long long lds, double* dst, long long ldd, int n,
                             int ncols, cudaStream_t s);

}  // namespace prrp
