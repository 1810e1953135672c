/*
 * prrp.h - C ABI of the GB300 (sm_103a) LU_PRRP library (libprrp.so).
 *
 * LU_PRRP is the blocked LU factorization with panel rank revealing pivoting of
 * Khabou, Demmel, Grigori and Gu (arXiv:1208.2451): every b-column panel is pivoted by a
 * strong rank revealing QR of its transpose (Section 2.1, Algorithm 1; Appendix A,
 * Algorithm 2), which bounds each block multiplier |L21| by tau and the growth factor by
 * (1 + tau b)^(n/b) (Section 2.2).
 *
 * Conventions for every entry point:
 *  - Matrices are ROW-MAJOR doubles: element (i, j) of a matrix with leading dimension ld
 *    is at p[i * ld + j]; ld >= number of columns.
 *  - Pointers named d* are device pointers owned by the caller (for example PyTorch
 *    tensors); pointers named h* are host pointers owned by the caller.  Handles
 *    (prrp_ctx, prrp_factors, prrp_server) are owned by the library and released with
 *    their destroy call.
 *  - "stream" is a cudaStream_t passed as void*; NULL means the legacy default stream.
 *    Work is enqueued in stream order.  Calls that return a device-side outcome
 *    (prrp_factor, prrp_solve, ...) synchronize the stream before they return.
 *  - Errors are reported only through return codes; nothing aborts or traps.  A kernel
 *    that meets an error (zero pivot, non-finite value, a wait that ran out) writes a
 *    status word and the kernels after it return at once.
 *  - One prrp_ctx per host thread.  The server object is internally locked.
 *  - The permutation convention is perm[i] = original row placed at position i, so
 *    (P A)[i, :] = A[perm[i], :] and P A = L U.
 */
#ifndef PRRP_H
#define PRRP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct prrp_ctx prrp_ctx;
typedef struct prrp_factors prrp_factors;

typedef enum {
  PRRP_OK = 0,
  PRRP_ERR_INVALID_ARG = 1,   /* bad size, pointer, leading dimension or option */
  PRRP_ERR_SINGULAR = 2,      /* zero pivot; stats.info holds its 1-based column */
  PRRP_ERR_NONFINITE = 3,     /* NaN or Inf in the input matrix */
  PRRP_ERR_OOM = 4,           /* device or host allocation failed */
  PRRP_ERR_CUDA = 5,          /* a CUDA runtime call failed */
  PRRP_ERR_TIMEOUT = 6,       /* a bounded device-side wait ran out */
  PRRP_ERR_SWAP_LIMIT = 7,    /* a panel needed more than opts.max_swaps interchanges */
  PRRP_ERR_NOT_CONVERGED = 8, /* iterative refinement stopped above its target */
  PRRP_ERR_BUSY = 9,          /* server: request can never fit the admission budget */
  PRRP_ERR_UNSUPPORTED = 10   /* size or option outside what the library supports */
} prrp_status;

typedef enum {
  PRRP_FP64 = 0,   /* Schur update and TRSM in FP64 (DFMA) */
  PRRP_TF32 = 1,   /* Schur update on tcgen05 tensor cores in TF32, FP32 accumulation */
  PRRP_BF16X3 = 2, /* Schur update on tcgen05 as 3-term split BF16, FP32 accumulation */
  PRRP_FP32 = 3,   /* FP32 factor (batched path) */
  PRRP_FP64_EMU = 4 /* Schur update to FP64 accuracy on the BF16 tensor cores: every operand
                       line cut into 8 signed base-128 digits under a power-of-two scale,
                       the 36 leading digit products accumulated exactly in FP32, assembled
                       exactly in 64-bit integers (b <= 64); the rest of the path in FP64 */
} prrp_precision;

typedef struct {
  int b;                /* panel width, 1 <= b <= 128 (default 64) */
  double tau;           /* strong RRQR threshold, tau >= 1 (default 2; the paper uses tau > 1) */
  int prec;             /* prrp_precision of the trailing update (default PRRP_FP64) */
  int max_swaps;        /* interchanges allowed per panel after QRCP (default 64) */
  int refine_max_iter;  /* FP64 iterative refinement corrections (default 10) */
  double refine_target; /* stop refining once eta <= target (default 2^-53) */
} prrp_opts;

typedef struct {
  double growth;   /* g_W = max(|A|, every block Schur complement A22 after an update) / max|A|
                      (Section 2.2: the entries after each block elimination step) */
  double growth_u; /* max |U| / max |A| (adds the diagonal-block GEPP) */
  double max_l21;  /* largest |block multiplier| (R11^-1 R12)^T over all panels, <= tau */
  double amax;     /* max |a_ij| of the input */
  int swaps;       /* strong RRQR interchanges over all panels */
  int info;        /* 1-based column of the first zero pivot, 0 if none */
  int panels;      /* panels factored */
} prrp_factor_stats;

typedef struct {
  int iterations;  /* correction solves: classic refinement steps + preconditioned GMRES steps */
  double eta0;     /* normwise backward error (1-norm) of the first solution */
  double eta;      /* normwise backward error of the returned solution */
} prrp_solve_info;

/* Fill *opts with the defaults above. */
void prrp_opts_default(prrp_opts* opts);

/* Human-readable name of a status code (static string). */
const char* prrp_status_string(prrp_status s);

/* Library version string (static). */
const char* prrp_version(void);

/* Text of the last CUDA failure seen by ctx (valid until the next call on ctx). */
const char* prrp_ctx_last_error(const prrp_ctx* ctx);

/* Create a context bound to CUDA device `device`.  It owns device workspace that grows
 * with the largest problem seen.  Returns INVALID_ARG for a bad device, CUDA otherwise. */
prrp_status prrp_create(prrp_ctx** ctx, int device);
prrp_status prrp_destroy(prrp_ctx* ctx);

/*
 * prrp_factor - LU_PRRP of the n x n row-major matrix dA (Algorithm 1).
 *
 * For each panel j (columns k0 .. k0+w-1, w = min(b, n-k0)):
 *   1. strong RRQR of the transposed panel selects w pivot rows (Algorithm 2: QR with
 *      column pivoting, then interchanges while some |(R11^-1 R12)_ij| > tau);
 *   2. L21 = (R11^-1 R12)^T (Algorithm 1, line 4);
 *   3. the row permutation is applied to all n columns (line 5);
 *   4. A22 -= L21 A12 (eq. "update", line 7);
 *   5. GEPP on the w x w diagonal block and U12 = L11^-1 Pi_jj^T A12 (lines 10-11);
 *   6. the rows below the block receive the final L21 Pi_jj L11, so that on return dA holds
 *      the ordinary unit-lower L (strictly below the diagonal) and U (on and above it).
 * With prec = PRRP_TF32 or PRRP_BF16X3, steps 4, 5 (U12, through an FP32 inverse of L11)
 * and 6 run on the tensor cores; the pivot choices of steps 1 and 5 stay FP64.  With
 * prec = PRRP_FP64_EMU only step 4 runs on the tensor cores, to FP64 accuracy (b <= 64,
 * UNSUPPORTED otherwise), and the factors serve like FP64 ones.
 * n = 0 is a no-op.  dA is overwritten; *F receives a handle holding the permutation and
 * statistics (and a reference to dA, which must stay alive while F is used).
 * Errors: INVALID_ARG, NONFINITE (checked before any write to dA), SINGULAR (dA then holds
 * a partial factorization), SWAP_LIMIT, TIMEOUT, CUDA, OOM, UNSUPPORTED (n > 65536 or
 * panel larger than the GPU's shared memory, or prec not available).
 */
prrp_status prrp_factor(prrp_ctx* ctx, int n, double* dA, int lda, const prrp_opts* opts,
                        void* stream, prrp_factors** F);

/*
 * prrp_factor_calu - CALU_PRRP (Section 3): prrp_factor with the panel pivots of step 1
 * chosen by tournament pivoting (Section 3.1) instead of one strong RRQR of the whole
 * panel.  The panel's rows are cut into leaves of leaf_rows rows (the last leaf takes the
 * remainder; a panel of fewer than 2 leaf_rows rows is one leaf); the strong RRQR of each
 * leaf's transpose selects w candidates, which lead their leaf; a binary tree then merges
 * consecutive nodes, left then right, by the strong RRQR of the 2w candidates, the
 * selected rows taking the left node's positions (an unpaired node goes up unchanged).
 * Each node's interchanges move whole rows.  L21 = (R11^-1 R12)^T then comes from the
 * unpivoted QR of the permuted panel, so |L21| is no longer bounded by tau; Section 3.2
 * bounds the growth by (1 + tau b)^((n/b)(H+1) - 1), H the height of the tree.  Steps 3
 * to 6 are those of prrp_factor, in every precision mode.  With one leaf per panel
 * (leaf_rows >= n) the pivots are those of prrp_factor.
 * Requires b <= 64 and b <= leaf_rows <= 128 (UNSUPPORTED for b > 64 or leaf_rows > 128,
 * INVALID_ARG for leaf_rows < max(b, 1)); the context keeps an n x n workspace for the row
 * moves.  Other arguments, outputs and errors as prrp_factor.
 */
prrp_status prrp_factor_calu(prrp_ctx* ctx, int n, double* dA, int lda, const prrp_opts* opts, int leaf_rows,
                             void* stream, prrp_factors** F);

/*
 * prrp_factor_block - block parallel (tree = 0) or block pairwise (tree = 1) LU_PRRP
 * (Section 5, algebra in Appendix E), for stability studies: the paper reports these
 * variants as less stable than LU_PRRP and CALU_PRRP.  Per panel the active rows are cut
 * into P' = max(1, min(blocks, m / (w + 1))) blocks of m / P' rows (the last takes the
 * remainder).  A tree of strong RRQRs runs over them: block parallel, a binary tree (a
 * merge node holds its children's selections, left then right); block pairwise, a flat
 * tree (node i holds the running selection and all rows of block i).  Each node's
 * permutation acts on its rows, so its selection leads; each row it does not select is
 * eliminated at once, A_e(k0+w:n) -= D_e A_sel(k0+w:n) with D = (R11^-1 R12)^T (|D| <= tau),
 * using rows not yet updated in this panel, and D_e is stored in the row's panel columns.
 * The root's w rows lead the active rows; GEPP on their diagonal block and
 * U12 = L11^-1 Pi_jj^T A12 follow.  On return dA holds those pivot rows' L11\U11 and U12,
 * every eliminated row's D in the panel's columns, and F the permutation and statistics
 * (growth = g_W over every updated row, max_l21 = max |D|).  The factorization is a
 * product of lower triangular factors, not P A = L U: prrp_solve returns UNSUPPORTED for
 * it.  FP64 only; b <= 64; every tree node must hold at most 255 rows (UNSUPPORTED
 * otherwise: use more blocks).  Other arguments and errors as prrp_factor.
 */
prrp_status prrp_factor_block(prrp_ctx* ctx, int n, double* dA, int lda, const prrp_opts* opts, int blocks,
                              int tree, void* stream, prrp_factors** F);

/* Copy the permutation (n ints, may be NULL) and statistics (may be NULL) to the host. */
prrp_status prrp_factors_get(const prrp_factors* F, int* hperm, prrp_factor_stats* stats);

/* Device pointer to the factor's permutation (n ints, library-owned). */
const int* prrp_factors_perm_device(const prrp_factors* F);

void prrp_factors_destroy(prrp_factors* F);

/*
 * prrp_solve - X = A^-1 B with the factors of prrp_factor (Section 2.3 solver tests):
 * Y = P B, forward substitution with the unit-lower L, back substitution with U.
 * dB (n x nrhs, row-major, ldb) is overwritten by X.  If dA_orig (the unfactored matrix,
 * n x n, lda of the factorization) is not NULL, FP64 iterative refinement follows
 * (Section 3.3): r = B - A X in FP64, X += (LU)^-1 P r, until eta <= opts.refine_target,
 * eta stops halving, or opts.refine_max_iter corrections (opts may be NULL: defaults).
 * Factors from a TF32 or BF16X3 Schur update are applied in FP32 for the corrections; when
 * such a correction lowers eta by less than 10x (ill-conditioned A), refinement continues
 * with GMRES on the system preconditioned by the factors ((LU)^-1 A d = (LU)^-1 r, FP64
 * except the preconditioner), restarted every 30 steps, at most opts.refine_max_iter
 * restart cycles.  NOT_CONVERGED when the limits are reached above the target.
 * info (may be NULL) receives eta of the first and final solutions (max over columns).
 */
prrp_status prrp_solve(prrp_ctx* ctx, const prrp_factors* F, const double* dA_orig, int nrhs,
                       double* dB, int ldb, const prrp_opts* opts, void* stream,
                       prrp_solve_info* info);

/*
 * prrp_gesv_host - end-to-end solve from HOST memory: copies hA (n x n, lda) and hB
 * (n x nrhs, ldb) to device workspace owned by ctx, factors, solves (refining in FP64
 * against the copied A when opts->refine_max_iter > 0), and copies X back into hX
 * (n x nrhs, ldb).  hA and hB are not modified.  Pinned host memory gives the fastest
 * copies; pageable memory works.
 */
prrp_status prrp_gesv_host(prrp_ctx* ctx, int n, const double* hA, int lda, int nrhs,
                           const double* hB, int ldb, double* hX, const prrp_opts* opts,
                           void* stream, prrp_factor_stats* stats, prrp_solve_info* info);

/*
 * prrp_batch_solve - solve `count` independent systems A_i X_i = B_i (n_i <= 1024) in one
 * persistent launch: one CTA runs the whole of Algorithm 1 (strong RRQR panels with tau
 * interchanges, Schur update, diagonal GEPP, U12, final L) on one system at a time, taking
 * systems largest first from a work list, then solves and refines in FP64 (Section 3.3).
 *
 * Host arrays of length count: n, lda, nrhs, ldb, and dA / dB (device pointers).  Each A_i
 * is an n_i x n_i row-major FP64 matrix (not modified); each B_i (n_i x nrhs_i, ldb_i) is
 * overwritten by X_i.  dPerm (host array of device pointers, may be NULL; entries may be
 * NULL) receives each system's row permutation (n_i ints, perm[i] = original row at i).
 * opts (may be NULL): b (<= 32, default 16 here), tau, max_swaps,
 * refine_max_iter, refine_target, prec = PRRP_FP32 (default: FP32 working copy and Schur
 * update, FP64 panel selection, GEPP, substitution arithmetic and residual) or PRRP_FP64.
 * per_system (host, count, may be NULL) receives each system's status; info (host, count,
 * may be NULL) its refinement count and first/final normwise backward error (max over its
 * right-hand sides).  Returns PRRP_OK when every system succeeded, otherwise the first
 * failing status in input order.  The launch shape (CTAs per SM x the update's register
 * tile) is tuned on first use of each (precision, b, size bucket of 128) and kept for the
 * process, per device; the launch sequence is replayed as a captured CUDA graph while the
 * batch shape is unchanged.
 */
prrp_status prrp_batch_solve(prrp_ctx* ctx, int count, const int* n, const double* const* dA,
                             const int* lda, const int* nrhs, double* const* dB, const int* ldb,
                             int* const* dPerm, const prrp_opts* opts, void* stream,
                             prrp_status* per_system, prrp_solve_info* info);

/*
 * prrp_batch_tune - tune prrp_batch_solve's launch shape ahead of use for every size
 * bucket of 128 up to nmax (<= 1024) under opts (may be NULL: the prrp_batch_solve
 * defaults), so that no batch waits on the tuning.  It times candidate shapes on a
 * synthetic sample (a few hundred MB of device memory for the largest bucket) on
 * `stream`; a shape already tuned in this process is not tuned again.  INVALID_ARG,
 * UNSUPPORTED (nmax > 1024 or prec other than FP32 / FP64), OOM, CUDA.
 */
prrp_status prrp_batch_tune(prrp_ctx* ctx, int nmax, const prrp_opts* opts, void* stream);

/* ---- serving: continuous batching of solve requests (serve.cpp) ---- */

typedef struct prrp_server prrp_server;

typedef struct {
  int n;              /* system size, >= 1 */
  int nrhs;           /* right-hand sides, >= 0 */
  const double* hA;   /* host, n x n row-major (lda), read until the request completes */
  int lda;
  const double* hB;   /* host, n x nrhs (ldb) */
  int ldb;
  double* hX;         /* host, n x nrhs (ldx): receives the solution */
  int ldx;
} prrp_request;

typedef struct {
  prrp_status status; /* the request's outcome */
  int iterations;     /* FP64 refinement corrections */
  double eta;         /* normwise backward error of the returned solution (max over RHS) */
  double latency_us;  /* submit to completion */
  double queue_us;    /* submit to admission */
} prrp_result;

typedef struct {
  uint64_t submitted, completed, rejected, units;
  double p50_us, p99_us, mean_us;   /* request latency percentiles (submit to completion) */
  double solves_per_s;              /* completed requests / (first submit .. last completion) */
  uint64_t peak_bytes_in_use;       /* largest admitted working set, <= the budget */
  int peak_busy_lanes;              /* most lanes with work on the device at once */
} prrp_serve_stats;

/*
 * prrp_server_create - start a serving loop on ctx's device with `lanes` worker lanes
 * (1..16; each lane owns a context and a stream, so lanes' work overlaps on the GPU) and
 * an HBM admission budget in bytes for the requests' device working sets.  A request is
 * admitted when its working set fits the budget left by the requests on the device;
 * the batched path's launch shapes are tuned during the call (prrp_batch_tune);
 * requests with n <= 512 that are admitted together are solved by one batched launch
 * (prrp_batch_solve); larger ones by prrp_factor + prrp_solve with their factors held in
 * device memory until their FP64 refinement ends.  opts (may be NULL): prec = PRRP_FP32
 * (default; FP32 batched factors, BF16X3 tensor-core Schur update for large n) or
 * PRRP_FP64; b, tau, max_swaps, refine_max_iter, refine_target as for prrp_factor.
 */
prrp_status prrp_server_create(prrp_ctx* ctx, size_t hbm_budget_bytes, const prrp_opts* opts, int lanes,
                               prrp_server** server);

/* Queue a request (non-blocking).  PRRP_ERR_BUSY if its working set can never fit the
 * budget.  *ticket identifies it for prrp_server_wait.  The host buffers must stay valid
 * until the wait returns. */
prrp_status prrp_server_submit(prrp_server* server, const prrp_request* req, uint64_t* ticket);

/* Block until the request completes (timeout_us < 0: no limit) and release its ticket.
 * PRRP_ERR_TIMEOUT if it did not complete in time (the ticket stays valid). */
prrp_status prrp_server_wait(prrp_server* server, uint64_t ticket, int64_t timeout_us, prrp_result* out);

prrp_status prrp_server_stats(prrp_server* server, prrp_serve_stats* stats);

/* Finish the queued requests, stop the lanes and free the server. */
prrp_status prrp_server_destroy(prrp_server* server);

/* Device a context is bound to. */
prrp_status prrp_ctx_device(const prrp_ctx* ctx, int* device);

/* ---- single steps of Algorithm 1, exposed for verification and measurement ---- */

/*
 * prrp_panel_select - steps 1-2 above on one m x w panel dP (row-major, ldp >= w),
 * 1 <= w <= min(m, 128): strong RRQR of dP^T (Algorithm 2).  On return
 *   hOrder[i] (m ints, host) = panel row placed at position i (positions 0..w-1 are the
 *             selected rows, in pivot order);
 *   dL21     ((m - w) x w, row-major, ld w, device) = (R11^-1 R12)^T, row i belonging to
 *             the panel row at position w + i;
 *   *hSwaps   = interchanges made after QRCP.
 * dP is not modified.  SINGULAR if the panel has rank < w, SWAP_LIMIT as above.
 */
prrp_status prrp_panel_select(prrp_ctx* ctx, int m, int w, const double* dP, int ldp,
                              double tau, int max_swaps, int* hOrder, double* dL21,
                              int* hSwaps, void* stream);

/*
 * prrp_schur_update - step 4 alone: C -= L * U with C m x n (ldc), L m x k (ldl),
 * U k x n (ldu), 1 <= k <= 128, all row-major device pointers, computed in `prec`
 * (PRRP_FP64 uses DFMA; PRRP_TF32 / PRRP_BF16X3 use tcgen05 with FP32 accumulation;
 * PRRP_FP64_EMU uses tcgen05 on exact BF16 digits for an FP64-accurate result, k <= 64).
 * In the tensor-core precisions C may alias L or U (the operands are split into the
 * context's workspace before C is written), which is how the factorization runs U12 and
 * the final multipliers (steps 5-6) on the tensor cores; in PRRP_FP64 they must not overlap.
 */
prrp_status prrp_schur_update(prrp_ctx* ctx, int m, int n, int k, const double* dL, int ldl,
                              const double* dU, int ldu, double* dC, int ldc, int prec,
                              void* stream);

/* Kernel classes for prrp_ctx_kernel_stats. */
enum {
  PRRP_KIND_SCAN = 0,     /* input scan and permutation init */
  PRRP_KIND_PANEL = 1,    /* strong RRQR panel (Algorithm 2) */
  PRRP_KIND_PERMUTE = 2,  /* row interchanges of the panel (Algorithm 1, line 5) */
  PRRP_KIND_UPDATE = 3,   /* Schur update A22 -= L21 A12 (line 7) */
  PRRP_KIND_DIAG = 4,     /* GEPP of the diagonal block (line 10) */
  PRRP_KIND_U12 = 5,      /* U12 = L11^-1 Pi_jj^T A12 and block-row interchanges (line 11) */
  PRRP_KIND_LFIX = 6,     /* final multipliers L21 Pi_jj L11 */
  PRRP_KIND_SOLVE = 7,    /* gather, forward/back substitution, refinement */
  PRRP_KIND_BATCH = 8,    /* the batched-solve kernel */
  PRRP_KIND_COUNT = 9
};

/* Enable (1) or disable (0) per-kernel-class timing: each launch of ctx is bracketed by
 * CUDA events on its stream and the elapsed times are summed per class after the call's
 * synchronize.  Launch and algorithmic-flop counters are kept whether or not it is on.
 * enable = 2 also keeps a launch timeline (see prrp_ctx_timeline), starting from an event
 * recorded in this call; any call to this function clears the timeline.  INVALID_ARG for
 * other values. */
prrp_status prrp_ctx_set_timing(prrp_ctx* ctx, int enable);

/* Panel kernel placement for this context (a tuning knob; results do not change).  Panels
 * (Algorithm 2 on an m x w panel) with m <= cluster_max_rows run as one thread-block
 * cluster of up to 16 CTAs that the hardware co-schedules, so panels of different
 * contexts or streams may run at the same time; taller panels run as one cooperative grid
 * over the SMs, and cooperative panels of one device run one at a time.  For a single
 * factorization the grid is faster above 512 rows; several factorizations sharing the GPU
 * (the serve loop) gain from clusters.  A cluster's CTAs hold m / 16 rows each above 512
 * rows; a panel whose rows do not fit a CTA's shared memory runs as a grid instead.
 * cluster_max_rows in [0, 4096], 0 = the default (512); INVALID_ARG otherwise. */
prrp_status prrp_ctx_set_panel_mode(prrp_ctx* ctx, int cluster_max_rows);

/* SM split of the tensor-core modes (PRRP_TF32, PRRP_BF16X3, PRRP_FP64_EMU) for this
 * context (a tuning knob; results do not change).  Their trailing-update kernels hold one
 * SM's shared memory per CTA, so a panel (Algorithm 2) cannot run on the SMs they hold.
 * prrp_factor in these modes therefore runs the panels, and the narrow update of the next
 * panel's columns between them, on at most panel_ctas CTAs (more when a panel's rows would
 * not fit them), the diagonal-block work (GEPP, U12, the final multipliers) on at most
 * block_ctas, and the rest of each trailing update on the remaining SMs, so that the
 * panel of step j + 1 runs beside the update of step j.  0 selects the library default
 * (64 and 8; 96 and 8 for PRRP_TF32 and PRRP_BF16X3 at n <= 10240, where the panels take
 * a larger share of the work); panel_ctas equal to the SM count turns the split off.
 * INVALID_ARG when a value is negative or above the SM count, or when the two leave fewer
 * than 8 SMs for the rest update.  The plain FP64 mode is not affected. */
prrp_status prrp_ctx_set_sm_split(prrp_ctx* ctx, int panel_ctas, int block_ctas);

/* Aggregated trailing update of prrp_factor in the modes PRRP_TF32 and PRRP_BF16X3
 * (Algorithm 1, line 7; a tuning knob, off by default).  The panels are grouped in blocks
 * of q = floor(nb / b) panels.  Inside a block, each panel's row interchanges, Schur update
 * and U12 reach only the block's own columns and the multipliers on its left; the columns
 * right of the block are brought up to date once at the block's end: the block's composed
 * row interchanges, U = L_blk^-1 X for the block's rows (L_blk the block's unit lower
 * triangle of final multipliers; solved panel by panel with the 3 x BF16 product) and one
 * rank-(q b) update A22 -= L2 U.  This equals the per-panel order up to rounding, since
 * each panel's update L21 A12 is its final multipliers times its U12 rows.  The pivots are
 * those of the updated matrix as before; the growth factor is then taken over the block's
 * own columns at every panel and over the rest at block ends.  nb in [0, 256]; 0 (the
 * default) and nb < 2 b keep the per-panel update.  INVALID_ARG otherwise.  Other modes
 * are not affected. */
prrp_status prrp_ctx_set_update_block(prrp_ctx* ctx, int nb);

/* Substitution form of prrp_solve for this context (a tuning knob).  mode 0 (the default):
 * a triangle with at most 16 right-hand sides is solved by one launch whose CTAs wait for
 * one another's row blocks, the lowest latency for one solve on an otherwise idle GPU;
 * mode 1: one launch per 64-row block, which holds no SM while it waits, for contexts that
 * share the GPU with other work.  The two differ only in the order of rounding.
 * INVALID_ARG for other modes. */
prrp_status prrp_ctx_set_solve_mode(prrp_ctx* ctx, int mode);

/* The launch timeline kept under timing level 2: for each timed launch, in the order the
 * calls collected them, its kernel class (PRRP_KIND_*) and its start and end in ms after
 * the base event.  Launches on different streams overlap when they ran concurrently.
 * Copies min(cap, total) entries into the host arrays kinds, t0_ms, t1_ms (each at least
 * cap long) and stores the total in *count. */
prrp_status prrp_ctx_timeline(prrp_ctx* ctx, int cap, int* kinds, double* t0_ms, double* t1_ms,
                              int* count);

/* Copy the per-class totals since the last reset (arrays of PRRP_KIND_COUNT; any may be
 * NULL): milliseconds (only while timing is on), kernel launches, algorithmic flops
 * (update: 2 (m-w)(n-k0-w) w per panel).  reset != 0 zeroes them afterwards. */
prrp_status prrp_ctx_kernel_stats(prrp_ctx* ctx, double* ms, long long* launches,
                                  long long* flops, int reset);

/*
 * prrp_panel_select_noalloc - prrp_panel_select for callers that cannot allocate device
 * memory.  The paper has no counterpart: it is a deployment variant of the same panel
 * kernel (same grid rule, same arithmetic, same outputs).
 *
 * Who needs it: code that runs inside a device-memory arena owned by another allocator,
 * where a side allocation can fail or fragment the arena; loops whose latency budget
 * cannot absorb the device synchronization cudaMalloc/cudaFree may imply; and code that
 * must not create a prrp_ctx (its workspace is allocated).  This call takes no context
 * and calls no cudaMalloc, cudaFree or other allocating routine.
 *
 * Scratch: the kernel's device state word and cross-CTA exchange records live in one
 * library-wide static device array of 2,014,976 bytes, which every GPU that loads libprrp.so
 * holds until the process exits.  The call runs on the caller's current device: dP,
 * dOrder and dL21 must be device memory of that device (INVALID_ARG otherwise).  All calls
 * share the array and it keeps the last call's contents (the state word and the exchange
 * flags are cleared at the start of each call): calls that overlap on the GPU, from any
 * stream or thread, race and must not be issued.
 *
 * Limits: the exchange records hold at most 160 CTAs (the grid is min(#SMs, 160,
 * ceil(m/32)) CTAs); a panel whose rows then exceed one CTA's shared memory returns
 * PRRP_ERR_UNSUPPORTED.  Arguments as prrp_panel_select, except dOrder (m ints, DEVICE,
 * caller-owned) receives the order; hSwaps (host, may be NULL) the interchange count.
 * The call synchronizes `stream` and reads the kernel's status on the host, so it cannot
 * be used inside stream capture.  It returns that status (SINGULAR, SWAP_LIMIT, TIMEOUT)
 * or INVALID_ARG / UNSUPPORTED / CUDA.
 */
prrp_status prrp_panel_select_noalloc(int m, int w, const double* dP, int ldp, double tau,
                                      int max_swaps, int* dOrder, double* dL21, int* hSwaps,
                                      void* stream);

/*
 * prrp_selftest_wait - check of the failure path of the device-side bounded waits (no
 * counterpart in the paper): launches a two-CTA cooperative grid in which one CTA waits at
 * a grid barrier that the other never reaches.  The wait gives up after `spin_limit` polls
 * (about 100 ns each; 0 = the library default of ~2 s) and the call returns
 * PRRP_ERR_TIMEOUT with the context still usable.  Any other return is a failure.
 */
prrp_status prrp_selftest_wait(prrp_ctx* ctx, unsigned spin_limit, void* stream);

/*
 * prrp_selftest_chain_wait - the same check for the one-launch substitution of prrp_solve
 * (no counterpart in the paper): one CTA holding the ticket of row block 1 of a two-block
 * triangle waits for block 0, which no CTA solves.  The wait gives up after `spin_limit`
 * polls (0 = the library default) and the call returns PRRP_ERR_TIMEOUT, with the
 * context still usable.  Any other return is a failure.
 */
prrp_status prrp_selftest_chain_wait(prrp_ctx* ctx, unsigned spin_limit, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PRRP_H */
