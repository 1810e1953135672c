// C ABI of libprrp.so: argument checks, device workspace, and the host-side loop of
// Algorithm 1 that enqueues one panel's kernels after another on the caller's stream.
// Every pivot decision stays on the device; the host reads the device state word once,
// after the last panel.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <numeric>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "prrp.h"

using namespace prrp;

namespace prrp {

cudaError_t smem_optin_ptr(const void* kernel) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, cudaError_t> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  auto it = done.find({dev, kernel});
  if (it != done.end()) return it->second;
  cudaFuncAttributes fa{};
  e = cudaFuncGetAttributes(&fa, kernel);
  int optin = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - static_cast<int>(fa.sharedSizeBytes));
  done[{dev, kernel}] = e;
  return e;
}

}  // namespace prrp

struct prrp_ctx {
  int device = 0;
  int num_sms = 0;
  size_t smem_optin = 0;
  DevState* st = nullptr;       // device
  double* xval = nullptr;       // panel exchange records
  int2* xkey = nullptr;
  double* xvec = nullptr;
  unsigned long long* qkey = nullptr;   // QRCP step keys [kQSlots][xcap][kQKeyStride]
  double* qrow = nullptr;               // QRCP records [kQSlots][xcap][kQStride]
  int xcap = 0;                 // CTAs the exchange can hold
  int* pairs = nullptr;
  int pairs_cap = 0;
  int* ipiv = nullptr;
  int* order = nullptr;
  int order_cap = 0;
  double* l21 = nullptr;        // (n - w) x w multipliers of the current panel
  size_t l21_cap = 0;
  double* solve_ws = nullptr;   // Y, R, B0 (n x nrhs each) and norms
  size_t solve_cap = 0;
  double* norms = nullptr;      // 3 * kMaxRhsNorms doubles + anorm
  int norms_cap = 0;
  double* hA = nullptr;         // prrp_gesv_host device copies
  size_t hA_cap = 0;
  double* hA0 = nullptr;
  size_t hA0_cap = 0;
  double* hB = nullptr;
  size_t hB_cap = 0;
  unsigned char* tcws = nullptr;    // split operands of the tensor-core update
  size_t tcws_cap = 0;
  // look-ahead: side streams, events, second multiplier buffer, A12 snapshots, second
  // tensor-core workspace
  cudaStream_t s_rest = nullptr, s_blk = nullptr;
  std::vector<cudaEvent_t> evs;
  size_t ev_next = 0;
  double* l21b = nullptr;
  size_t l21b_cap = 0;
  double* a12 = nullptr;            // two snapshots of the block row right of the panel
  size_t a12_cap = 0;
  unsigned char* tcws2 = nullptr;
  size_t tcws2_cap = 0;
  unsigned char* tcws3 = nullptr;   // tensor-core workspace of the block stream (a7)
  size_t tcws3_cap = 0;
  double* tri = nullptr;            // I - L11^-1 and I - L11 of the current panel
  size_t tri_cap = 0;
  // substitution: inverted diagonal blocks (FP64 and FP32), FP32 copy of the factors, the
  // factorization they were made from (generation number), step counters
  double* dinv64 = nullptr;
  size_t dinv64_cap = 0;
  unsigned long long dinv64_gen = 0;
  float* dinv32 = nullptr;
  size_t dinv32_cap = 0;
  float* lu32 = nullptr;
  size_t lu32_cap = 0;
  unsigned long long lu32_gen = 0;
  float* y32 = nullptr;
  size_t y32_cap = 0;
  unsigned* tcount = nullptr;       // substitution counters; word 0: a chain wait that ran out
  size_t tcount_cap = 0;
  double* zbuf = nullptr;           // second n x nrhs buffer of the one-launch substitution
  size_t zbuf_cap = 0;
  int panel_cluster_rows = 0;       // prrp_ctx_set_panel_mode (0: the library default)
  int split_panel = 0;              // prrp_ctx_set_sm_split (0: the library defaults)
  int split_blk = 0;
  int solve_mode = 0;               // prrp_ctx_set_solve_mode
  int agg_nb = 0;                   // prrp_ctx_set_update_block (0: per-panel update)
  // aggregated update of the mixed-precision forms: row order at the block's start, where
  // each row sat then, the moved rows and their count, the moves' buffers for the next
  // block's columns and for the rest
  int* agg_perm0 = nullptr;
  int* agg_pos0 = nullptr;
  int* agg_pairs = nullptr;
  size_t agg_perm0_cap = 0, agg_pos0_cap = 0, agg_pairs_cap = 0;
  double* agg_tmp1 = nullptr;
  double* agg_tmp2 = nullptr;
  size_t agg_tmp1_cap = 0, agg_tmp2_cap = 0;
  cudaEvent_t agg_ev[3] = {};       // the block's end on s; the far update's splits; its end
  double* krylov = nullptr;         // GMRES-based refinement: Krylov basis, coefficients
  size_t krylov_cap = 0;
  double* gm_coef = nullptr;
  size_t gm_coef_cap = 0;
  int* calu_pmap = nullptr;         // CALU_PRRP: tournament position -> panel row
  int* calu_ptmp = nullptr;         //   row moves through tmp
  double* calu_tmp = nullptr;
  size_t calu_cap = 0;              //   rows of n doubles the tmp holds (n of the factorization)
  unsigned* gemm_ctr = nullptr;     // tile counters of the FP64 updates (critical, rest stream)
  size_t gemm_ctr_cap = 0;
  unsigned long long factor_gen = 0;
  // batched solves: metadata, per-CTA workspace, outputs, tuned launch shapes, graphs
  unsigned char* bmeta = nullptr;
  size_t bmeta_cap = 0;
  unsigned char* bws = nullptr;
  size_t bws_cap = 0;
  unsigned char* bout = nullptr;
  size_t bout_cap = 0;
  std::map<long long, int> batch_tuned;     // (fp64, b, size bucket) -> 4 * CTAs per SM + tile rows
  struct BatchGraph { cudaGraphExec_t exec = nullptr; std::vector<long long> sig; };
  BatchGraph bgraph;
  cudaStream_t capture_stream = nullptr;
  std::string last_error;
  // optional per-kernel-class timing with CUDA events on the launching stream
  bool timing = false;
  struct Rec { cudaEvent_t a, b; int kind; };
  std::vector<Rec> recs;
  size_t nrec = 0;
  double kind_ms[PRRP_KIND_COUNT] = {};
  // optional launch timeline (timing level 2): (kind, start, end) in ms after tl_base
  cudaEvent_t tl_base = nullptr;
  struct Span { int kind; float t0, t1; };
  std::vector<Span> timeline;
  long long kind_launches[PRRP_KIND_COUNT] = {};
  long long kind_flops[PRRP_KIND_COUNT] = {};
};

struct prrp_factors {
  prrp_ctx* ctx = nullptr;
  int n = 0;
  double* dA = nullptr;
  long long lda = 0;
  int* perm = nullptr;          // device, owned
  prrp_factor_stats stats{};
  prrp_opts opts{};
  unsigned long long gen = 0;   // identifies this factorization to the context's solve caches
  int kind = 0;                 // 0: P A = L U; 1: block LU_PRRP's product form (no prrp_solve)
};

namespace {

// Wraps one kernel launch: counts it and, when timing is on, brackets it with events.
struct Timed {
  prrp_ctx* ctx;
  cudaStream_t s;
  size_t idx = (size_t)-1;
  Timed(prrp_ctx* c, cudaStream_t st, int kind, long long flops = 0) : ctx(c), s(st) {
    ctx->kind_launches[kind] += 1;
    ctx->kind_flops[kind] += flops;
    if (!ctx->timing) return;
    if (ctx->nrec == ctx->recs.size()) {
      prrp_ctx::Rec r{};
      cudaEventCreate(&r.a);
      cudaEventCreate(&r.b);
      ctx->recs.push_back(r);
    }
    idx = ctx->nrec++;
    ctx->recs[idx].kind = kind;
    cudaEventRecord(ctx->recs[idx].a, s);
  }
  ~Timed() {
    if (idx != (size_t)-1) cudaEventRecord(ctx->recs[idx].b, s);
  }
};

// After a synchronize: fold the recorded event pairs into per-kind totals.
void collect_timing(prrp_ctx* ctx) {
  for (size_t i = 0; i < ctx->nrec; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->recs[i].a, ctx->recs[i].b) == cudaSuccess)
      ctx->kind_ms[ctx->recs[i].kind] += ms;
    float t0 = 0.f, t1 = 0.f;       // timeline: the launch's interval after the base event
    if (ctx->tl_base && cudaEventElapsedTime(&t0, ctx->tl_base, ctx->recs[i].a) == cudaSuccess &&
        cudaEventElapsedTime(&t1, ctx->tl_base, ctx->recs[i].b) == cudaSuccess)
      ctx->timeline.push_back({ctx->recs[i].kind, t0, t1});
  }
  ctx->nrec = 0;
}

prrp_status cuda_fail(prrp_ctx* ctx, cudaError_t e, const char* what) {
  if (ctx) ctx->last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? PRRP_ERR_OOM : PRRP_ERR_CUDA;
}

#define CK(call)                                              \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e, #call);  \
  } while (0)

template <typename T>
prrp_status grow(prrp_ctx* ctx, T** p, size_t* cap, size_t need) {
  if (need <= *cap && *p) return PRRP_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  size_t want = std::max<size_t>(need, 1);
  cudaError_t e = cudaMalloc((void**)p, want * sizeof(T));
  if (e != cudaSuccess) { *p = nullptr; return cuda_fail(ctx, e, "cudaMalloc"); }
  *cap = want;
  return PRRP_OK;
}

template <typename T>
prrp_status grow_i(prrp_ctx* ctx, T** p, int* cap, int need) {
  size_t c = (size_t)*cap;
  prrp_status s = grow(ctx, p, &c, (size_t)need);
  *cap = (int)c;
  return s;
}

double bits_to_double(unsigned long long b) {
  double d;
  std::memcpy(&d, &b, sizeof d);
  return d;
}

prrp_status check_opts(const prrp_opts* o) {
  if (o->b < 1 || o->b > kMaxW) return PRRP_ERR_INVALID_ARG;
  if (!(o->tau >= 1.0)) return PRRP_ERR_INVALID_ARG;
  if (o->max_swaps < 0) return PRRP_ERR_INVALID_ARG;
  if (o->prec < PRRP_FP64 || o->prec > PRRP_FP64_EMU) return PRRP_ERR_INVALID_ARG;
  if (o->refine_max_iter < 0) return PRRP_ERR_INVALID_ARG;
  return PRRP_OK;
}

// Cooperative grid size for an m-row panel: <= one CTA per SM (and <= kPanelMaxCtas),
// >= 32 rows per CTA, and <= max_ctas when that is given, unless the rows per CTA would
// then not fit a CTA's shared memory.
prrp_status panel_grid(prrp_ctx* ctx, int m, int w, int* G, int* rpc, int max_ctas = 0) {
  const int gmax = std::min(ctx->num_sms, kPanelMaxCtas);
  int g = std::max(1, std::min(gmax, (m + 31) / 32));
  if (max_ctas > 0) g = std::min(g, max_ctas);
  int r = (m + g - 1) / g;
  // the kernel's static shared memory (under 8 KB) comes out of the same opt-in limit
  const size_t limit = ctx->smem_optin - 8192;
  while (panel_smem_for(w, r) > limit && g < gmax) {
    ++g;
    r = (m + g - 1) / g;
  }
  if (panel_smem_for(w, r) > limit) return PRRP_ERR_UNSUPPORTED;
  *G = g;
  *rpc = r;
  return PRRP_OK;
}

prrp_status ensure_panel_ws(prrp_ctx* ctx, int n, int w, int max_swaps) {
  prrp_status s;
  if (ctx->xcap < kPanelMaxCtas) {
    const int G = kPanelMaxCtas;
    size_t c1 = 0, c2 = 0, c3 = 0, c4 = 0, c5 = 0;
    if (ctx->xval) { cudaFree(ctx->xval); cudaFree(ctx->xkey); cudaFree(ctx->xvec); }
    if (ctx->qkey) { cudaFree(ctx->qkey); cudaFree(ctx->qrow); }
    ctx->xval = nullptr; ctx->xkey = nullptr; ctx->xvec = nullptr; ctx->qkey = nullptr; ctx->qrow = nullptr;
    if ((s = grow(ctx, &ctx->xval, &c1, 2 * (size_t)G * kXVal)) != PRRP_OK) return s;
    if ((s = grow(ctx, &ctx->xkey, &c2, 2 * (size_t)G)) != PRRP_OK) return s;
    if ((s = grow(ctx, &ctx->xvec, &c3, 2 * (size_t)G * kMaxW)) != PRRP_OK) return s;
    if ((s = grow(ctx, &ctx->qkey, &c4, kQSlots * (size_t)G * kQKeyStride)) != PRRP_OK) return s;
    if ((s = grow(ctx, &ctx->qrow, &c5, kQSlots * (size_t)G * kQStride)) != PRRP_OK) return s;
    ctx->xcap = G;
  }
  if ((s = grow_i(ctx, &ctx->pairs, &ctx->pairs_cap, 4 * (w + max_swaps) + 8)) != PRRP_OK) return s;
  if ((s = grow(ctx, &ctx->l21, &ctx->l21_cap, (size_t)std::max(n, 1) * w)) != PRRP_OK) return s;
  if (!ctx->ipiv) CK(cudaMalloc(&ctx->ipiv, kMaxW * sizeof(int)));
  return PRRP_OK;
}

// Enqueue one panel's strong RRQR on rows [0, m) of the strip P (ldp): resets the barrier
// and the pair counter first.
prrp_status enqueue_panel(prrp_ctx* ctx, const double* P, long long ldp, int m, int w, double tau,
                          int max_swaps, int col_offset, double* L21, int ldl, int* order,
                          int* pairs, cudaStream_t s, int max_ctas = 0, int nopivot = 0) {
  int G = 0, rpc = 0;
  prrp_status ps = panel_grid(ctx, m, w, &G, &rpc, max_ctas);
  if (ps != PRRP_OK) return ps;
  CK(cudaMemsetAsync(&ctx->st->barrier, 0, 2 * sizeof(unsigned), s));
  // a QRCP key is absent while it holds 0 and a record word while it holds the sentinel;
  // the kernel prepares a slot itself only for its second use within the launch
  CK(cudaMemsetAsync(ctx->qkey, 0, kQSlots * sizeof(unsigned long long) * G * kQKeyStride, s));
  CK(cudaMemsetAsync(ctx->qrow, kQSentinelByte, kQSlots * sizeof(double) * G * kQStride, s));
  PanelParams p{};
  p.P = P; p.ldp = ldp; p.m = m; p.w = w; p.tau = tau; p.max_swaps = max_swaps;
  p.col_offset = col_offset; p.L21 = L21; p.ldl = ldl; p.order = order; p.pairs = pairs;
  p.st = ctx->st; p.xval = ctx->xval; p.xkey = ctx->xkey; p.xvec = ctx->xvec; p.rows_per_cta = rpc;
  p.qkey = ctx->qkey; p.qrow = ctx->qrow;
  p.nopivot = nopivot;
  p.cluster_rows = ctx->panel_cluster_rows;
  cudaError_t e = launch_panel(p, G, s);
  if (e == cudaErrorCooperativeLaunchTooLarge) return PRRP_ERR_UNSUPPORTED;
  if (e != cudaSuccess) return cuda_fail(ctx, e, "panel launch");
  return PRRP_OK;
}

// A recorded event from a small ring (record then wait is safe to reuse: a wait captures
// the event's state when it is enqueued).
cudaEvent_t next_event(prrp_ctx* ctx) {
  if (ctx->evs.empty()) {
    ctx->evs.resize(64);
    for (auto& e : ctx->evs) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  }
  cudaEvent_t e = ctx->evs[ctx->ev_next % ctx->evs.size()];
  ++ctx->ev_next;
  return e;
}

prrp_status read_state(prrp_ctx* ctx, DevState* h, cudaStream_t s) {
  CK(cudaMemcpyAsync(h, ctx->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return PRRP_OK;
}

}  // namespace

extern "C" {

void prrp_opts_default(prrp_opts* o) {
  if (!o) return;
  o->b = 64;
  o->tau = 2.0;
  o->prec = PRRP_FP64;
  o->max_swaps = 64;
  o->refine_max_iter = 10;
  o->refine_target = std::ldexp(1.0, -53);
}

const char* prrp_status_string(prrp_status s) {
  switch (s) {
    case PRRP_OK: return "ok";
    case PRRP_ERR_INVALID_ARG: return "invalid argument";
    case PRRP_ERR_SINGULAR: return "singular (zero pivot)";
    case PRRP_ERR_NONFINITE: return "non-finite input";
    case PRRP_ERR_OOM: return "out of memory";
    case PRRP_ERR_CUDA: return "CUDA error";
    case PRRP_ERR_TIMEOUT: return "device wait timed out";
    case PRRP_ERR_SWAP_LIMIT: return "strong RRQR swap limit reached";
    case PRRP_ERR_NOT_CONVERGED: return "refinement did not converge";
    case PRRP_ERR_BUSY: return "request exceeds admission budget";
    case PRRP_ERR_UNSUPPORTED: return "unsupported size or option";
  }
  return "unknown status";
}

const char* prrp_version(void) { return "prrp 0.1 (sm_103a)"; }

const char* prrp_ctx_last_error(const prrp_ctx* ctx) {
  return ctx ? ctx->last_error.c_str() : "no context";
}

prrp_status prrp_create(prrp_ctx** out, int device) {
  if (!out) return PRRP_ERR_INVALID_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
    return PRRP_ERR_INVALID_ARG;
  prrp_ctx* ctx = new (std::nothrow) prrp_ctx();
  if (!ctx) return PRRP_ERR_OOM;
  ctx->device = device;
  prrp_status st = PRRP_OK;
  do {
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) { st = cuda_fail(ctx, e, "cudaSetDevice"); break; }
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    ctx->num_sms = v;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    ctx->smem_optin = (size_t)v;
    cudaDeviceGetAttribute(&v, cudaDevAttrCooperativeLaunch, device);
    if (!v) { st = PRRP_ERR_UNSUPPORTED; break; }
    e = cudaMalloc(&ctx->st, sizeof(DevState));
    if (e != cudaSuccess) { st = cuda_fail(ctx, e, "cudaMalloc"); break; }
    cudaMemset(ctx->st, 0, sizeof(DevState));
  } while (0);
  if (st != PRRP_OK) { prrp_destroy(ctx); return st; }
  *out = ctx;
  return PRRP_OK;
}

prrp_status prrp_destroy(prrp_ctx* ctx) {
  if (!ctx) return PRRP_OK;
  cudaSetDevice(ctx->device);
  for (auto& r : ctx->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  if (ctx->tl_base) cudaEventDestroy(ctx->tl_base);
  if (ctx->bgraph.exec) cudaGraphExecDestroy(ctx->bgraph.exec);
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  if (ctx->bmeta) cudaFree(ctx->bmeta);
  if (ctx->bws) cudaFree(ctx->bws);
  if (ctx->bout) cudaFree(ctx->bout);
  void* ptrs[] = {ctx->st, ctx->xval, ctx->xkey, ctx->xvec, ctx->qkey, ctx->qrow, ctx->pairs, ctx->ipiv, ctx->order,
                  ctx->l21, ctx->solve_ws, ctx->norms, ctx->hA, ctx->hA0, ctx->hB, ctx->tcws,
                  ctx->l21b, ctx->a12, ctx->tcws2, ctx->dinv64, ctx->dinv32, ctx->lu32, ctx->y32,
                  ctx->tcount, ctx->zbuf, ctx->gemm_ctr, ctx->krylov, ctx->gm_coef, ctx->tcws3, ctx->tri,
                  ctx->calu_pmap, ctx->calu_ptmp, ctx->calu_tmp, ctx->agg_perm0, ctx->agg_pos0,
                  ctx->agg_pairs, ctx->agg_tmp1, ctx->agg_tmp2};
  for (cudaEvent_t e : ctx->evs) cudaEventDestroy(e);
  for (cudaEvent_t e : ctx->agg_ev)
    if (e) cudaEventDestroy(e);
  if (ctx->s_rest) cudaStreamDestroy(ctx->s_rest);
  if (ctx->s_blk) cudaStreamDestroy(ctx->s_blk);
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete ctx;
  return PRRP_OK;
}

}  // extern "C"

namespace {

// Algorithm 1 (leaf_rows == 0: LU_PRRP) or CALU_PRRP (Section 3.1: panel pivots from a
// tournament over leaves of leaf_rows rows, then L21 from an unpivoted QR of the panel).
prrp_status factor_impl(prrp_ctx* ctx, int n, double* dA, int lda, const prrp_opts* opts_in,
                        int leaf_rows, void* stream, prrp_factors** F) {
  if (!ctx || !F) return PRRP_ERR_INVALID_ARG;
  *F = nullptr;
  prrp_opts o;
  prrp_opts_default(&o);
  if (opts_in) o = *opts_in;
  if (n < 0 || lda < std::max(n, 1) || (n > 0 && !dA)) return PRRP_ERR_INVALID_ARG;
  prrp_status ps = check_opts(&o);
  if (ps != PRRP_OK) return ps;
  if (o.prec == PRRP_FP32 || (o.prec == PRRP_FP64_EMU && o.b > 64)) return PRRP_ERR_UNSUPPORTED;
  if (leaf_rows < 0 || (leaf_rows > 0 && leaf_rows < o.b)) return PRRP_ERR_INVALID_ARG;
  if (leaf_rows > 0 && (o.b > 64 || leaf_rows > 128)) return PRRP_ERR_UNSUPPORTED;
  if (n > 65536) return PRRP_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaSetDevice(ctx->device));

  prrp_factors* f = new (std::nothrow) prrp_factors();
  if (!f) return PRRP_ERR_OOM;
  f->ctx = ctx; f->n = n; f->dA = dA; f->lda = lda; f->opts = o; f->gen = ++ctx->factor_gen;
  auto fail = [&](prrp_status st) { prrp_factors_destroy(f); return st; };
  cudaError_t e = cudaMalloc(&f->perm, sizeof(int) * std::max(n, 1));
  if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "cudaMalloc perm"));
  if (n == 0) { f->stats.growth = f->stats.growth_u = 1.0; *F = f; return PRRP_OK; }

  const int b = std::min(o.b, n);
  if ((ps = ensure_panel_ws(ctx, n, b, o.max_swaps)) != PRRP_OK) return fail(ps);
  if (o.prec != PRRP_FP64 &&
      (ps = grow(ctx, &ctx->tcws, &ctx->tcws_cap, tc_workspace_bytes(o.prec, n, n, b))) != PRRP_OK)
    return fail(ps);
  {
    int G, rpc;   // the first panel is the tallest
    if ((ps = panel_grid(ctx, n, b, &G, &rpc)) != PRRP_OK) return fail(ps);
  }
  e = cudaMemsetAsync(ctx->st, 0, sizeof(DevState), s);
  if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "memset state"));
  {
    Timed t(ctx, s, PRRP_KIND_SCAN);
    if ((e = launch_iota(f->perm, n, s)) != cudaSuccess) return fail(cuda_fail(ctx, e, "iota"));
  }
  {
    Timed t(ctx, s, PRRP_KIND_SCAN);
    if ((e = launch_scan(dA, lda, n, ctx->st, s)) != cudaSuccess) return fail(cuda_fail(ctx, e, "scan"));
  }

  const int max_pairs = 2 * (b + o.max_swaps) + 2;
  // Look-ahead schedule.  Critical stream s: panel(j), permute(j), snapshot of the block
  // row A12 right of the panel, the narrow update of the next panel's columns; stream
  // s_rest: the rest of the update; stream s_blk: GEPP of the diagonal block, U12 and the
  // final multipliers.  permute(j+1) moves whole rows below the block, so it waits for
  // the rest update and the multipliers of panel j.  The updates read L21 from the panel's
  // own buffer (two alternate) and A12 from the snapshot, so U12 may overwrite A12 while
  // they run.
  if (!ctx->s_rest) {
    if ((e = cudaStreamCreateWithFlags(&ctx->s_rest, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&ctx->s_blk, cudaStreamNonBlocking)) != cudaSuccess)
      return fail(cuda_fail(ctx, e, "stream create"));
  }
  if ((ps = grow(ctx, &ctx->l21b, &ctx->l21b_cap, (size_t)n * b)) != PRRP_OK) return fail(ps);
  if (leaf_rows > 0 && ctx->calu_cap < (size_t)n) {
    // the tournament's row moves go through an n x n buffer (the first panel moves rows of
    // all n columns)
    size_t c1 = 0, c2 = 0, c3 = 0;
    if (ctx->calu_tmp) { cudaFree(ctx->calu_tmp); cudaFree(ctx->calu_pmap); cudaFree(ctx->calu_ptmp); }
    ctx->calu_tmp = nullptr; ctx->calu_pmap = nullptr; ctx->calu_ptmp = nullptr; ctx->calu_cap = 0;
    if ((ps = grow(ctx, &ctx->calu_tmp, &c1, (size_t)n * n)) != PRRP_OK) return fail(ps);
    if ((ps = grow(ctx, &ctx->calu_pmap, &c2, (size_t)n)) != PRRP_OK) return fail(ps);
    if ((ps = grow(ctx, &ctx->calu_ptmp, &c3, (size_t)n)) != PRRP_OK) return fail(ps);
    ctx->calu_cap = n;
  }
  if ((ps = grow(ctx, &ctx->a12, &ctx->a12_cap, 2 * (size_t)n * b)) != PRRP_OK) return fail(ps);
  if (o.prec != PRRP_FP64 &&
      (ps = grow(ctx, &ctx->tcws2, &ctx->tcws2_cap, tc_workspace_bytes(o.prec, n, b, b))) != PRRP_OK)
    return fail(ps);
  // a7 on the tensor cores in the low-precision modes: U12 (w x nc) and the multipliers
  // ((m - w) x w) share one workspace on the block stream
  const bool tc_a7 = o.prec == PRRP_TF32 || o.prec == PRRP_BF16X3;
  if (tc_a7) {
    const size_t ws3 = std::max(tc_workspace_bytes(o.prec, b, n, b), tc_workspace_bytes(o.prec, n, b, b));
    if ((ps = grow(ctx, &ctx->tcws3, &ctx->tcws3_cap, ws3)) != PRRP_OK) return fail(ps);
    if ((ps = grow(ctx, &ctx->tri, &ctx->tri_cap, 2 * (size_t)b * b)) != PRRP_OK) return fail(ps);
  }
  // Aggregated update (mixed-precision LU_PRRP, opt-in): blocks of q_agg panels whose row
  // moves, updates and U12 stay inside the block's columns; the columns right of a block
  // are moved, solved and updated once at its end, by one rank-NB product.
  int q_agg = 1;
  if (tc_a7 && leaf_rows == 0) q_agg = std::max(1, std::min(ctx->agg_nb, kAggMaxNB) / b);
  const int NB = q_agg * b;
  const bool agg = q_agg > 1 && n > NB;
  int agg_cap = 0;            // rows a block can move: its permutes' pairs and GEPP's rows
  if (agg) {
    agg_cap = (int)std::min<long long>(n, (long long)q_agg * (max_pairs + b));
    if ((ps = grow(ctx, &ctx->agg_perm0, &ctx->agg_perm0_cap, (size_t)n)) != PRRP_OK ||
        (ps = grow(ctx, &ctx->agg_pos0, &ctx->agg_pos0_cap, (size_t)n)) != PRRP_OK ||
        (ps = grow(ctx, &ctx->agg_pairs, &ctx->agg_pairs_cap, 2 * (size_t)agg_cap + 1)) != PRRP_OK ||
        (ps = grow(ctx, &ctx->agg_tmp1, &ctx->agg_tmp1_cap, (size_t)agg_cap * NB)) != PRRP_OK ||
        (ps = grow(ctx, &ctx->agg_tmp2, &ctx->agg_tmp2_cap, (size_t)agg_cap * n)) != PRRP_OK ||
        (ps = grow(ctx, &ctx->tri, &ctx->tri_cap, 2 * (size_t)q_agg * 2 * b * b)) != PRRP_OK)
      return fail(ps);
    const size_t w2s = std::max({tc_workspace_bytes(o.prec, n, NB, b), tc_workspace_bytes(PRRP_BF16X3, b, NB, NB),
                                 tc_workspace_bytes(o.prec, n, NB, NB)});
    const size_t wrs = std::max(tc_workspace_bytes(PRRP_BF16X3, b, n, NB), tc_workspace_bytes(o.prec, n, n, NB));
    if ((ps = grow(ctx, &ctx->tcws2, &ctx->tcws2_cap, w2s)) != PRRP_OK ||
        (ps = grow(ctx, &ctx->tcws, &ctx->tcws_cap, wrs)) != PRRP_OK)
      return fail(ps);
    for (cudaEvent_t& ev : ctx->agg_ev)
      if (!ev && (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
        return fail(cuda_fail(ctx, e, "event create"));
  }
  cudaStream_t sr = ctx->s_rest, sb = ctx->s_blk;
  cudaEvent_t ev_start = next_event(ctx);
  CK(cudaEventRecord(ev_start, s));
  CK(cudaStreamWaitEvent(sr, ev_start, 0));
  CK(cudaStreamWaitEvent(sb, ev_start, 0));
  cudaEvent_t ev_rest = nullptr, ev_blk = nullptr;        // of the previous panel
  // C (mm x nn) -= L (mm x kk, ld kk) * U (kk x nn, ld ldu)
  if ((ps = grow(ctx, &ctx->gemm_ctr, &ctx->gemm_ctr_cap, 2)) != PRRP_OK) return fail(ps);
  // SM split of the tensor-core modes.  Their update kernels hold a whole SM's shared memory
  // per CTA, so a panel cannot share an SM with them: the panels (and the narrow update
  // between them, on the same stream) get split_panel SMs, the block stream's kernels
  // split_blk, and the rest update the others.  The FP64 update shares SMs with the panels
  // and keeps the whole GPU.
  int cap_panel = 0, cap_blk = 0, cap_rest = 0;
  if (o.prec != PRRP_FP64) {
    const bool small_n = n <= kSplitSmallN && o.prec != PRRP_FP64_EMU;
    cap_panel = ctx->split_panel > 0 ? ctx->split_panel : (small_n ? kSplitPanelSmallN : kSplitPanelDefault);
    cap_blk = ctx->split_blk > 0 ? ctx->split_blk : kSplitBlkDefault;
    if (cap_panel >= ctx->num_sms) {
      cap_panel = cap_blk = 0;                 // no split: every kernel may take every SM
    } else {
      cap_rest = std::max(8, ctx->num_sms - cap_panel - cap_blk);
    }
  }
  auto update = [&](int mm, int nn, int kk, const double* L, const double* U, long long ldu, double* C,
                    unsigned char* ws, cudaStream_t st) -> cudaError_t {
    if (o.prec == PRRP_FP64)   // one tile counter per stream: the narrow and rest updates overlap
      return launch_gemm_fp64(mm, nn, kk, L, kk, U, ldu, C, lda, ctx->st, 1, ctx->num_sms, st, 1,
                              ctx->gemm_ctr + (st == sr ? 1 : 0));
    ctx->kind_launches[PRRP_KIND_UPDATE] += 2;   // the two operand splits before the MMA kernel
    return launch_tc_update(o.prec, mm, nn, kk, L, kk, U, ldu, C, lda, ctx->st, 1, ws, st,
                            st == sr ? cap_rest : cap_panel);
  };
  int K0 = 0, KB = n;                                      // the current block's columns
  cudaEvent_t ev_split = nullptr, ev_far = nullptr;        // far update of the previous block
  for (int jp = 0, k0 = 0; k0 < n; k0 += b, ++jp) {
    const int w = std::min(b, n - k0), m = n - k0;
    const int w2 = std::min(b, n - k0 - w);                 // next panel's width (0: last)
    double* Akk = dA + (long long)k0 * lda + k0;
    double* L21 = (jp & 1) ? ctx->l21b : ctx->l21;
    double* A12 = ctx->a12 + (size_t)(jp & 1) * n * b;     // snapshot: w x nc, ld nc
    const bool blk_first = agg && jp % q_agg == 0;
    if (blk_first) {
      K0 = k0;
      KB = std::min(n, k0 + NB);
      // the row order at the block's start (rows above K0 are no longer moved)
      CK(cudaMemcpyAsync(ctx->agg_perm0, f->perm + k0, sizeof(int) * (n - k0), cudaMemcpyDeviceToDevice, s));
    }
    const bool blk_last = agg && k0 + w >= KB;
    const int ncol = agg ? KB : n;                         // columns the panel's moves and U12 reach
    // I - L11^-1 and I - L11 of this panel: kept for the block's end in the aggregated form
    // (two sets of q_agg panels, alternating by block)
    double* tri = agg ? ctx->tri + ((size_t)((jp / q_agg) & 1) * q_agg + jp % q_agg) * 2 * b * b : ctx->tri;
    if (leaf_rows == 0) {
      {
        Timed t(ctx, s, PRRP_KIND_PANEL, 3LL * m * w * w);
        ps = enqueue_panel(ctx, Akk, lda, m, w, o.tau, o.max_swaps, k0, L21, w, nullptr, ctx->pairs, s, cap_panel);
      }
      if (ps != PRRP_OK) return fail(ps);
      if (ev_rest) CK(cudaStreamWaitEvent(s, ev_rest, 0));
      if (ev_blk) CK(cudaStreamWaitEvent(s, ev_blk, 0));
      // the previous block's far update has taken its multipliers (rows this block moves)
      if (blk_first && ev_split) CK(cudaStreamWaitEvent(s, ev_split, 0));
    } else {
      // CALU_PRRP: the tournament reads only the panel's columns; its row moves (whole
      // rows) wait for the rest update and the block work of the previous panel; then
      // L21 from the unpivoted QR of the permuted panel (no row moves of its own).
      TournParams tp{};
      tp.P = Akk; tp.ldp = lda; tp.m = m; tp.w = w; tp.leaf = leaf_rows;
      tp.nleaf = std::max(1, m / leaf_rows);
      int h = 0;
      while ((1 << h) < tp.nleaf) ++h;
      tp.height = h;
      tp.mode = 0; tp.level0 = 0; tp.level1 = h + 1;      // the whole tree in one launch
      tp.tau = o.tau; tp.max_swaps = o.max_swaps; tp.col_offset = k0; tp.pmap = ctx->calu_pmap; tp.st = ctx->st;
      {
        Timed t(ctx, s, PRRP_KIND_PANEL, 3LL * m * w * w);
        e = launch_iota(ctx->calu_pmap, m, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(&ctx->st->barrier, 0, sizeof(unsigned), s);
        if (e == cudaSuccess) e = launch_tournament(tp, std::min(ctx->num_sms, kPanelMaxCtas), s);
      }
      if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "tournament"));
      if (ev_rest) CK(cudaStreamWaitEvent(s, ev_rest, 0));
      if (ev_blk) CK(cudaStreamWaitEvent(s, ev_blk, 0));
      {
        Timed t(ctx, s, PRRP_KIND_PERMUTE);
        e = launch_gather_permute(dA, lda, n, k0, m, ctx->calu_pmap, f->perm, ctx->calu_tmp, ctx->calu_ptmp,
                                  ctx->st, s);
      }
      if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "tournament row moves"));
      {
        Timed t(ctx, s, PRRP_KIND_PANEL, 3LL * m * w * w);
        ps = enqueue_panel(ctx, Akk, lda, m, w, o.tau, o.max_swaps, k0, L21, w, nullptr, ctx->pairs, s, cap_panel,
                           1);
      }
      if (ps != PRRP_OK) return fail(ps);
    }
    {
      Timed t(ctx, s, PRRP_KIND_PERMUTE);
      e = launch_permute(dA, lda, ncol, k0, ctx->pairs, max_pairs, f->perm, ctx->st, s);
    }
    if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "permute"));
    cudaEvent_t ev_perm = next_event(ctx);
    CK(cudaEventRecord(ev_perm, s));
    // block diagonal work on s_blk: GEPP now, U12 and the multipliers after the snapshot
    CK(cudaStreamWaitEvent(sb, ev_perm, 0));
    {
      Timed t(ctx, sb, PRRP_KIND_DIAG, 2LL * w * w * w / 3);
      e = launch_diag_gepp(dA, lda, k0, w, ctx->ipiv, f->perm, ctx->st, sb);
    }
    if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "diag gepp"));
    const int nc = ncol - k0 - w;                           // columns right of the panel updated now
    if (m > w && agg) {
      // every update of the block's own columns at once, on the critical stream
      if (nc > 0)
        CK(cudaMemcpy2DAsync(A12, sizeof(double) * nc, Akk + w, sizeof(double) * lda, sizeof(double) * nc, w,
                             cudaMemcpyDeviceToDevice, s));
      cudaEvent_t ev_snap = next_event(ctx);
      CK(cudaEventRecord(ev_snap, s));
      if (nc > 0) {
        Timed t(ctx, s, PRRP_KIND_UPDATE, 2LL * (m - w) * nc * w);
        e = update(m - w, nc, w, L21, A12, nc, Akk + (long long)w * lda + w, ctx->tcws2, s);
      }
      if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "schur update (block columns)"));
      CK(cudaStreamWaitEvent(sb, ev_snap, 0));
    } else if (m > w) {
      CK(cudaMemcpy2DAsync(A12, sizeof(double) * nc, Akk + w, sizeof(double) * lda, sizeof(double) * nc, w,
                           cudaMemcpyDeviceToDevice, s));
      cudaEvent_t ev_snap = next_event(ctx);
      CK(cudaEventRecord(ev_snap, s));
      {
        Timed t(ctx, s, PRRP_KIND_UPDATE, 2LL * (m - w) * w2 * w);
        e = update(m - w, w2, w, L21, A12, nc, Akk + (long long)w * lda + w, ctx->tcws2, s);
      }
      if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "schur update (next panel)"));
      if (nc > w2) {
        CK(cudaStreamWaitEvent(sr, ev_snap, 0));
        {
          Timed t(ctx, sr, PRRP_KIND_UPDATE, 2LL * (m - w) * (nc - w2) * w);
          e = update(m - w, nc - w2, w, L21, A12 + w2, nc, Akk + (long long)w * lda + w + w2, ctx->tcws, sr);
        }
        if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "schur update"));
        ev_rest = next_event(ctx);
        CK(cudaEventRecord(ev_rest, sr));
      }
      CK(cudaStreamWaitEvent(sb, ev_snap, 0));
    }
    if (tc_a7 && n > w) {
      // U12 = X - (I - L11^-1) X and (L21 Pi_jj) L11 = Y - Y (I - L11) on the tensor cores
      {
        Timed t(ctx, sb, PRRP_KIND_U12, 1LL * nc * w * w);
        ctx->kind_launches[PRRP_KIND_U12] += nc > 0 ? 4 : 1;   // swaps, E, 2 splits, MMA
        e = launch_u12(dA, lda, ncol, k0, w, ctx->ipiv, ctx->st, sb, 0);
        if (e == cudaSuccess) e = launch_tri_blocks(dA, lda, k0, w, tri, ctx->st, sb);
        if (e == cudaSuccess && nc > 0)
          e = launch_tc_update(o.prec, w, nc, w, tri, w, Akk + w, lda, Akk + w, lda, ctx->st, 2,
                               ctx->tcws3, sb, cap_blk);
      }
      if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "u12"));
      if (m > w) {
        Timed t(ctx, sb, PRRP_KIND_LFIX, 1LL * (m - w) * w * w);
        double* Y = Akk + (long long)w * lda;
        ctx->kind_launches[PRRP_KIND_LFIX] += 3;               // copy, 2 splits, MMA
        e = launch_lfix_copy(dA, lda, n, k0, w, L21, w, ctx->ipiv, ctx->st, sb);
        if (e == cudaSuccess)
          e = launch_tc_update(o.prec, m - w, w, w, Y, lda, tri + (size_t)w * w, w, Y, lda, ctx->st, 0,
                               ctx->tcws3, sb, cap_blk);
      }
      if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "lfix"));
    } else {
      if (n > w) {
        Timed t(ctx, sb, PRRP_KIND_U12, 1LL * nc * w * w);
        e = launch_u12(dA, lda, n, k0, w, ctx->ipiv, ctx->st, sb);
      }
      if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "u12"));
      if (m > w) {
        Timed t(ctx, sb, PRRP_KIND_LFIX, 1LL * (m - w) * w * w);
        e = launch_lfix(dA, lda, n, k0, w, L21, w, ctx->ipiv, ctx->st, sb);
      }
      if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "lfix"));
    }
    ev_blk = next_event(ctx);
    CK(cudaEventRecord(ev_blk, sb));
    if (blk_last && KB < n) {
      // the block's end: the columns right of it (next block's first, on the critical
      // stream; the rest on s_rest, beside the next block's panels)
      const int nF = n - KB, nF1 = std::min(NB, nF), nF2 = nF - nF1;
      double* L2 = dA + (long long)KB * lda + K0;           // final multipliers below the block
      int* cnt = ctx->agg_pairs + 2 * (size_t)agg_cap;
      const double* tri_set = ctx->tri + (size_t)((jp / q_agg) & 1) * q_agg * 2 * b * b;
      // U(K0:KB, c0:c0+nc) = L_blk^-1 A(K0:KB, c0:c0+nc), panel by panel: the rows of panel t
      // lose the earlier panels' part (final multipliers times their U rows), then take
      // L11^-1 as X - (I - L11^-1) X, as the per-panel U12 does.  These U rows are operands
      // of the rank-NB update (the per-panel form updates with the unreduced A12 instead),
      // so they are formed with the FP32-accurate 3 x BF16 product in both modes.
      const int uprec = PRRP_BF16X3;
      auto block_u = [&](int c0, int nc, unsigned char* ws, cudaStream_t st, int cap) -> cudaError_t {
        cudaError_t r = cudaSuccess;
        for (int t = 0; t < q_agg && r == cudaSuccess; ++t) {
          double* Xt = dA + (long long)(K0 + t * b) * lda + c0;
          if (t > 0) {
            ctx->kind_launches[PRRP_KIND_U12] += 3;
            r = launch_tc_update(uprec, b, nc, t * b, dA + (long long)(K0 + t * b) * lda + K0, lda,
                                 dA + (long long)K0 * lda + c0, lda, Xt, lda, ctx->st, 1, ws, st, cap);
          }
          if (r == cudaSuccess) {
            ctx->kind_launches[PRRP_KIND_U12] += 3;
            r = launch_tc_update(uprec, b, nc, b, tri_set + (size_t)t * 2 * b * b, b, Xt, lda, Xt, lda, ctx->st, 2,
                                 ws, st, cap);
          }
        }
        return r;
      };
      CK(cudaStreamWaitEvent(s, ev_blk, 0));
      if (ev_far) CK(cudaStreamWaitEvent(s, ev_far, 0));    // the previous far update wrote these
      {
        Timed t(ctx, s, PRRP_KIND_PERMUTE);
        ctx->kind_launches[PRRP_KIND_PERMUTE] += 3;          // positions, pairs, gather, scatter
        e = launch_block_pairs(ctx->agg_perm0, f->perm, K0, n - K0, ctx->agg_pos0, ctx->agg_pairs, cnt, agg_cap,
                               ctx->st, s);
        if (e == cudaSuccess)
          e = launch_block_moves(dA, lda, K0, KB, nF1, ctx->agg_pairs, cnt, agg_cap, ctx->agg_tmp1, ctx->st, s);
      }
      if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "block row moves"));
      {
        Timed t(ctx, s, PRRP_KIND_U12, 1LL * NB * nF1 * NB);
        ctx->kind_launches[PRRP_KIND_U12] -= 1;
        e = block_u(KB, nF1, ctx->tcws2, s, cap_panel);
      }
      if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "block U12"));
      {
        Timed t(ctx, s, PRRP_KIND_UPDATE, 2LL * (n - KB) * nF1 * NB);
        ctx->kind_launches[PRRP_KIND_UPDATE] += 2;
        e = launch_tc_update(o.prec, n - KB, nF1, NB, L2, lda, dA + (long long)K0 * lda + KB, lda,
                             dA + (long long)KB * lda + KB, lda, ctx->st, 1, ctx->tcws2, s, cap_panel);
      }
      if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "block update"));
      ev_split = ev_far = nullptr;
      if (nF2 > 0) {
        const int c2 = KB + nF1;
        CK(cudaEventRecord(ctx->agg_ev[0], s));
        CK(cudaStreamWaitEvent(sr, ctx->agg_ev[0], 0));
        {
          Timed t(ctx, sr, PRRP_KIND_PERMUTE);
          ctx->kind_launches[PRRP_KIND_PERMUTE] += 1;
          e = launch_block_moves(dA, lda, K0, c2, nF2, ctx->agg_pairs, cnt, agg_cap, ctx->agg_tmp2, ctx->st, sr);
        }
        if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "block row moves (rest)"));
        {
          Timed t(ctx, sr, PRRP_KIND_U12, 1LL * NB * nF2 * NB);
          ctx->kind_launches[PRRP_KIND_U12] -= 1;
          e = block_u(c2, nF2, ctx->tcws, sr, cap_rest);
        }
        if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "block U12 (rest)"));
        {
          Timed t(ctx, sr, PRRP_KIND_UPDATE, 2LL * (n - KB) * nF2 * NB);
          ctx->kind_launches[PRRP_KIND_UPDATE] += 2;
          e = launch_tc_update(o.prec, n - KB, nF2, NB, L2, lda, dA + (long long)K0 * lda + c2, lda,
                               dA + (long long)KB * lda + c2, lda, ctx->st, 1, ctx->tcws, sr, cap_rest,
                               ctx->agg_ev[1]);
        }
        if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "block update (rest)"));
        ev_split = ctx->agg_ev[1];
        ev_far = ctx->agg_ev[2];
        CK(cudaEventRecord(ev_far, sr));
      }
    }
  }
  if (ev_rest) CK(cudaStreamWaitEvent(s, ev_rest, 0));
  if (ev_blk) CK(cudaStreamWaitEvent(s, ev_blk, 0));
  if (ev_far) CK(cudaStreamWaitEvent(s, ev_far, 0));
  DevState h{};
  if ((ps = read_state(ctx, &h, s)) != PRRP_OK) return fail(ps);
  collect_timing(ctx);
  f->stats.amax = bits_to_double(h.amax_bits);
  f->stats.growth = f->stats.amax > 0 ? bits_to_double(h.gmax_bits) / f->stats.amax : 1.0;
  f->stats.growth_u = f->stats.amax > 0 ? bits_to_double(h.umax_bits) / f->stats.amax : 1.0;
  f->stats.max_l21 = bits_to_double(h.l21_bits);
  f->stats.swaps = h.swaps_total;
  f->stats.info = h.info;
  f->stats.panels = (n + b - 1) / b;
  *F = f;
  if (h.status != 0) {
    if (h.status == PRRP_ERR_TIMEOUT) {
      char buf[64];
      std::snprintf(buf, sizeof buf, "device wait at site %u ran out", h.timeout_site);
      ctx->last_error = buf;
    }
    return (prrp_status)h.status;
  }
  return PRRP_OK;
}

}  // namespace

extern "C" {

prrp_status prrp_factor(prrp_ctx* ctx, int n, double* dA, int lda, const prrp_opts* opts_in,
                        void* stream, prrp_factors** F) {
  return factor_impl(ctx, n, dA, lda, opts_in, 0, stream, F);
}

prrp_status prrp_factor_block(prrp_ctx* ctx, int n, double* dA, int lda, const prrp_opts* opts_in, int blocks,
                              int tree, void* stream, prrp_factors** F) {
  if (!ctx || !F) return PRRP_ERR_INVALID_ARG;
  *F = nullptr;
  prrp_opts o;
  prrp_opts_default(&o);
  if (opts_in) o = *opts_in;
  if (n < 0 || lda < std::max(n, 1) || (n > 0 && !dA) || blocks < 1 || (tree != 0 && tree != 1))
    return PRRP_ERR_INVALID_ARG;
  prrp_status ps = check_opts(&o);
  if (ps != PRRP_OK) return ps;
  if (o.prec != PRRP_FP64 || o.b > 64 || n > 65536) return PRRP_ERR_UNSUPPORTED;
  const int b = std::min(o.b, std::max(n, 1));
  // every tree node must fit one CTA: the largest block (the last one) plus, for the flat
  // tree, the running selection
  for (int k0 = 0; k0 < n; k0 += b) {
    const int w = std::min(b, n - k0), m = n - k0;
    const int parts = std::max(1, std::min(blocks, m / (w + 1)));
    const int q = m / parts, last = m - (parts - 1) * q;
    const int rows = std::max(tree == 1 && parts > 1 ? w + last : last, parts > 1 ? 2 * w : 0);
    if (rows > kTreeNodeMaxRows) return PRRP_ERR_UNSUPPORTED;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaSetDevice(ctx->device));
  prrp_factors* f = new (std::nothrow) prrp_factors();
  if (!f) return PRRP_ERR_OOM;
  f->ctx = ctx; f->n = n; f->dA = dA; f->lda = lda; f->opts = o; f->gen = ++ctx->factor_gen; f->kind = 1;
  auto fail = [&](prrp_status st) { prrp_factors_destroy(f); return st; };
  cudaError_t e = cudaMalloc(&f->perm, sizeof(int) * std::max(n, 1));
  if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "cudaMalloc perm"));
  if (n == 0) { f->stats.growth = f->stats.growth_u = 1.0; *F = f; return PRRP_OK; }
  if ((ps = ensure_panel_ws(ctx, n, b, o.max_swaps)) != PRRP_OK) return fail(ps);
  if (ctx->calu_cap < (size_t)n) {
    size_t c1 = 0, c2 = 0, c3 = 0;
    if (ctx->calu_tmp) { cudaFree(ctx->calu_tmp); cudaFree(ctx->calu_pmap); cudaFree(ctx->calu_ptmp); }
    ctx->calu_tmp = nullptr; ctx->calu_pmap = nullptr; ctx->calu_ptmp = nullptr; ctx->calu_cap = 0;
    if ((ps = grow(ctx, &ctx->calu_tmp, &c1, (size_t)n * n)) != PRRP_OK) return fail(ps);
    if ((ps = grow(ctx, &ctx->calu_pmap, &c2, (size_t)n)) != PRRP_OK) return fail(ps);
    if ((ps = grow(ctx, &ctx->calu_ptmp, &c3, (size_t)n)) != PRRP_OK) return fail(ps);
    ctx->calu_cap = n;
  }
  if ((e = cudaMemsetAsync(ctx->st, 0, sizeof(DevState), s)) != cudaSuccess) return fail(cuda_fail(ctx, e, "memset"));
  if ((e = launch_iota(f->perm, n, s)) != cudaSuccess) return fail(cuda_fail(ctx, e, "iota"));
  if ((e = launch_scan(dA, lda, n, ctx->st, s)) != cudaSuccess) return fail(cuda_fail(ctx, e, "scan"));
  const int sms = std::min(ctx->num_sms, kPanelMaxCtas);
  for (int k0 = 0; k0 < n; k0 += b) {
    const int w = std::min(b, n - k0), m = n - k0;
    const int parts = std::max(1, std::min(blocks, m / (w + 1)));
    int height = 0;
    if (tree == 0) while ((1 << height) < parts) ++height;
    else height = parts - 1;
    double* Akk = dA + (long long)k0 * lda + k0;
    TournParams tp{};
    tp.P = Akk; tp.Pw = Akk; tp.ldp = lda; tp.m = m; tp.w = w; tp.leaf = m / parts; tp.nleaf = parts;
    tp.height = height; tp.mode = tree == 0 ? 1 : 2; tp.tau = o.tau; tp.max_swaps = o.max_swaps;
    tp.col_offset = k0; tp.pmap = ctx->calu_pmap; tp.st = ctx->st;
    {
      Timed t(ctx, s, PRRP_KIND_PANEL, 3LL * m * w * w);
      e = launch_iota(ctx->calu_pmap, m, s);
      // each level: the nodes' selections (panel columns only), then their eliminations
      for (int h = 0; h <= height && e == cudaSuccess; ++h) {
        tp.level0 = h;
        tp.level1 = h + 1;
        e = launch_tournament(tp, sms, s);
        if (e == cudaSuccess) e = launch_tree_eliminate(tp, dA, lda, n, k0, sms, s);
      }
    }
    if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "block tree"));
    {
      Timed t(ctx, s, PRRP_KIND_PERMUTE);
      e = launch_gather_permute(dA, lda, n, k0, m, ctx->calu_pmap, f->perm, ctx->calu_tmp, ctx->calu_ptmp,
                                ctx->st, s);
    }
    if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "block row moves"));
    {
      Timed t(ctx, s, PRRP_KIND_DIAG, 2LL * w * w * w / 3);
      e = launch_diag_gepp(dA, lda, k0, w, ctx->ipiv, f->perm, ctx->st, s);
    }
    if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "diag gepp"));
    if (n > w) {
      Timed t(ctx, s, PRRP_KIND_U12, 1LL * (n - k0 - w) * w * w);
      e = launch_u12(dA, lda, n, k0, w, ctx->ipiv, ctx->st, s);
    }
    if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "u12"));
  }
  DevState h{};
  if ((ps = read_state(ctx, &h, s)) != PRRP_OK) return fail(ps);
  collect_timing(ctx);
  f->stats.amax = bits_to_double(h.amax_bits);
  f->stats.growth = f->stats.amax > 0 ? bits_to_double(h.gmax_bits) / f->stats.amax : 1.0;
  f->stats.growth_u = f->stats.amax > 0 ? bits_to_double(h.umax_bits) / f->stats.amax : 1.0;
  f->stats.max_l21 = bits_to_double(h.l21_bits);
  f->stats.swaps = h.swaps_total;
  f->stats.info = h.info;
  f->stats.panels = (n + b - 1) / b;
  *F = f;
  return h.status != 0 ? (prrp_status)h.status : PRRP_OK;
}

prrp_status prrp_factor_calu(prrp_ctx* ctx, int n, double* dA, int lda, const prrp_opts* opts, int leaf_rows,
                             void* stream, prrp_factors** F) {
  if (leaf_rows < 1) {
    if (F) *F = nullptr;
    return PRRP_ERR_INVALID_ARG;
  }
  return factor_impl(ctx, n, dA, lda, opts, leaf_rows, stream, F);
}

prrp_status prrp_factors_get(const prrp_factors* F, int* hperm, prrp_factor_stats* stats) {
  if (!F) return PRRP_ERR_INVALID_ARG;
  if (stats) *stats = F->stats;
  if (hperm && F->n > 0) {
    if (cudaSetDevice(F->ctx->device) != cudaSuccess) return PRRP_ERR_CUDA;
    if (cudaMemcpy(hperm, F->perm, sizeof(int) * F->n, cudaMemcpyDeviceToHost) != cudaSuccess)
      return PRRP_ERR_CUDA;
  }
  return PRRP_OK;
}

const int* prrp_factors_perm_device(const prrp_factors* F) { return F ? F->perm : nullptr; }

void prrp_factors_destroy(prrp_factors* F) {
  if (!F) return;
  if (F->perm) {
    cudaSetDevice(F->ctx->device);
    cudaFree(F->perm);
  }
  delete F;
}

// Inverted diagonal blocks (and for FP32 the FP32 copy of L\U) of factorization F, made
// on first use and kept in the context until another factorization is solved.
static prrp_status prepare_solve(prrp_ctx* ctx, const prrp_factors* F, bool fp32, cudaStream_t s) {
  const int n = F->n, nb = (n + 63) / 64;
  cudaError_t e;
  const size_t words = trsv_counter_words(n);
  if (ctx->tcount_cap < words) {
    prrp_status ps = grow(ctx, &ctx->tcount, &ctx->tcount_cap, words);
    if (ps != PRRP_OK) return ps;
    CK(cudaMemsetAsync(ctx->tcount, 0, sizeof(unsigned) * words, s));
  }
  prrp_status ps;
  if (!fp32) {
    if (ctx->dinv64_gen == F->gen) return PRRP_OK;
    if ((ps = grow(ctx, &ctx->dinv64, &ctx->dinv64_cap, (size_t)2 * nb * 4096)) != PRRP_OK) return ps;
    Timed t(ctx, s, PRRP_KIND_SOLVE, 2LL * nb * 64 * 64 * 64 / 3);
    if ((e = launch_invert_diag(F->dA, F->lda, n, ctx->dinv64, 0, s)) != cudaSuccess) return cuda_fail(ctx, e, "invert");
    ctx->dinv64_gen = F->gen;
    return PRRP_OK;
  }
  if (ctx->lu32_gen == F->gen) return PRRP_OK;
  if ((ps = grow(ctx, &ctx->dinv32, &ctx->dinv32_cap, (size_t)2 * nb * 4096)) != PRRP_OK) return ps;
  if ((ps = grow(ctx, &ctx->lu32, &ctx->lu32_cap, (size_t)n * n)) != PRRP_OK) return ps;
  {
    Timed t(ctx, s, PRRP_KIND_SOLVE, 2LL * nb * 64 * 64 * 64 / 3);
    if ((e = launch_invert_diag(F->dA, F->lda, n, ctx->dinv32, 1, s)) != cudaSuccess) return cuda_fail(ctx, e, "invert");
  }
  {
    Timed t(ctx, s, PRRP_KIND_SOLVE);
    if ((e = launch_convert_lu32(F->dA, F->lda, n, ctx->lu32, s)) != cudaSuccess) return cuda_fail(ctx, e, "convert");
  }
  ctx->lu32_gen = F->gen;
  return PRRP_OK;
}

// Waits for the stream; a one-launch substitution whose wait ran out has left the wait's
// site in counter word 0, which is reported (PRRP_ERR_TIMEOUT) and cleared.
static prrp_status sync_solve(prrp_ctx* ctx, cudaStream_t s) {
  unsigned site = 0;
  if (ctx->tcount) CK(cudaMemcpyAsync(&site, ctx->tcount, sizeof site, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (site == 0) return PRRP_OK;
  CK(cudaMemsetAsync(ctx->tcount, 0, sizeof site, s));
  char buf[64];
  std::snprintf(buf, sizeof buf, "substitution wait at site %u ran out", site);
  ctx->last_error = buf;
  return PRRP_ERR_TIMEOUT;
}

// Y = U^-1 L^-1 P B in FP64.
static prrp_status solve_into(prrp_ctx* ctx, const prrp_factors* F, const double* B, long long ldb,
                              int nrhs, double* Y, cudaStream_t s) {
  cudaError_t e;
  prrp_status ps = prepare_solve(ctx, F, false, s);
  if (ps != PRRP_OK) return ps;
  const int nb = (F->n + 63) / 64;
  const bool chain = nrhs <= kChainRhs && ctx->solve_mode == 0;
  if (chain && (ps = grow(ctx, &ctx->zbuf, &ctx->zbuf_cap, (size_t)F->n * nrhs)) != PRRP_OK) return ps;
  Timed t(ctx, s, PRRP_KIND_SOLVE, 2LL * F->n * F->n * nrhs);
  ctx->kind_launches[PRRP_KIND_SOLVE] += chain ? 2 : 2LL * nb;   // with the gather: 1 + 2 (or 2 nb) launches
  if ((e = launch_gather_rows(B, ldb, F->perm, F->n, nrhs, Y, s)) != cudaSuccess) return cuda_fail(ctx, e, "gather");
  if (chain) {
    if ((e = launch_trsv_chain(F->dA, F->lda, ctx->dinv64, F->n, Y, ctx->zbuf, nrhs, 1, 0, ctx->tcount, ctx->st,
                               s)) != cudaSuccess)
      return cuda_fail(ctx, e, "trsv L");
    if ((e = launch_trsv_chain(F->dA, F->lda, ctx->dinv64, F->n, ctx->zbuf, Y, nrhs, 0, 0, ctx->tcount, ctx->st,
                               s)) != cudaSuccess)
      return cuda_fail(ctx, e, "trsv U");
    return PRRP_OK;
  }
  if ((e = launch_trsv(F->dA, F->lda, ctx->dinv64, F->n, Y, nrhs, 1, 0, ctx->tcount + 1, s)) != cudaSuccess)
    return cuda_fail(ctx, e, "trsv L");
  if ((e = launch_trsv(F->dA, F->lda, ctx->dinv64, F->n, Y, nrhs, 0, 0, ctx->tcount + 1, s)) != cudaSuccess)
    return cuda_fail(ctx, e, "trsv U");
  return PRRP_OK;
}

// ctx->y32 = U^-1 L^-1 P B in FP32 arithmetic (B rounded to FP32).
static prrp_status solve_into32(prrp_ctx* ctx, const prrp_factors* F, const double* B, long long ldb, int nrhs,
                                cudaStream_t s) {
  cudaError_t e;
  prrp_status ps = prepare_solve(ctx, F, true, s);
  if (ps != PRRP_OK) return ps;
  if ((ps = grow(ctx, &ctx->y32, &ctx->y32_cap, (size_t)F->n * nrhs)) != PRRP_OK) return ps;
  const int nb = (F->n + 63) / 64;
  const bool chain = nrhs <= kChainRhs && ctx->solve_mode == 0;
  if (chain && (ps = grow(ctx, &ctx->zbuf, &ctx->zbuf_cap, ((size_t)F->n * nrhs + 1) / 2)) != PRRP_OK) return ps;
  float* z32 = reinterpret_cast<float*>(ctx->zbuf);
  Timed t(ctx, s, PRRP_KIND_SOLVE, 2LL * F->n * F->n * nrhs);
  ctx->kind_launches[PRRP_KIND_SOLVE] += chain ? 2 : 2LL * nb;
  if ((e = launch_gather_rows32(B, ldb, F->perm, F->n, nrhs, ctx->y32, s)) != cudaSuccess)
    return cuda_fail(ctx, e, "gather");
  if (chain) {
    if ((e = launch_trsv_chain(ctx->lu32, F->n, ctx->dinv32, F->n, ctx->y32, z32, nrhs, 1, 1, ctx->tcount, ctx->st,
                               s)) != cudaSuccess)
      return cuda_fail(ctx, e, "trsv L");
    if ((e = launch_trsv_chain(ctx->lu32, F->n, ctx->dinv32, F->n, z32, ctx->y32, nrhs, 0, 1, ctx->tcount, ctx->st,
                               s)) != cudaSuccess)
      return cuda_fail(ctx, e, "trsv U");
    return PRRP_OK;
  }
  if ((e = launch_trsv(ctx->lu32, F->n, ctx->dinv32, F->n, ctx->y32, nrhs, 1, 1, ctx->tcount + 1, s)) != cudaSuccess)
    return cuda_fail(ctx, e, "trsv L");
  if ((e = launch_trsv(ctx->lu32, F->n, ctx->dinv32, F->n, ctx->y32, nrhs, 0, 1, ctx->tcount + 1, s)) != cudaSuccess)
    return cuda_fail(ctx, e, "trsv U");
  return PRRP_OK;
}

prrp_status prrp_solve(prrp_ctx* ctx, const prrp_factors* F, const double* dA_orig, int nrhs,
                       double* dB, int ldb, const prrp_opts* opts_in, void* stream,
                       prrp_solve_info* info) {
  if (!ctx || !F || nrhs < 0 || ldb < std::max(nrhs, 1) || (F->n > 0 && nrhs > 0 && !dB))
    return PRRP_ERR_INVALID_ARG;
  prrp_opts o = F->opts;
  if (opts_in) {
    o.refine_max_iter = opts_in->refine_max_iter;
    o.refine_target = opts_in->refine_target;
  }
  if (info) { info->iterations = 0; info->eta0 = -1.0; info->eta = -1.0; }
  if (F->kind != 0) return PRRP_ERR_UNSUPPORTED;
  const int n = F->n;
  if (n == 0 || nrhs == 0) return PRRP_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaSetDevice(ctx->device));
  const size_t blk = (size_t)n * nrhs;
  prrp_status ps = grow(ctx, &ctx->solve_ws, &ctx->solve_cap, 3 * blk);
  if (ps != PRRP_OK) return ps;
  ps = grow_i(ctx, &ctx->norms, &ctx->norms_cap, 3 * nrhs + 1);
  if (ps != PRRP_OK) return ps;
  double* Y = ctx->solve_ws;
  double* R = Y + blk;
  double* B0 = R + blk;
  const bool refine = dA_orig != nullptr;
  // factors from a low-precision Schur update are only about FP32-accurate: with the FP64
  // residual of the refinement, FP32 substitution converges as fast and costs far less
  const bool low = refine && (F->opts.prec == PRRP_TF32 || F->opts.prec == PRRP_BF16X3);
  if (refine) CK(launch_copy_rows(dB, ldb, B0, nrhs, n, nrhs, s));
  if (low) {
    if ((ps = solve_into32(ctx, F, dB, ldb, nrhs, s)) != PRRP_OK) return ps;
    Timed t(ctx, s, PRRP_KIND_SOLVE);
    CK(cudaMemset2DAsync(dB, sizeof(double) * ldb, 0, sizeof(double) * nrhs, n, s));
    CK(launch_axpy_rows32(dB, ldb, ctx->y32, 1.0, n, nrhs, s));
  } else {
    if ((ps = solve_into(ctx, F, dB, ldb, nrhs, Y, s)) != PRRP_OK) return ps;
    Timed t(ctx, s, PRRP_KIND_SOLVE);
    CK(launch_copy_rows(Y, nrhs, dB, ldb, n, nrhs, s));
  }
  if (!refine) {
    ps = sync_solve(ctx, s);
    collect_timing(ctx);
    return ps;
  }
  double* anorm = ctx->norms + 3 * nrhs;
  CK(launch_norm1(dA_orig, F->lda, n, anorm, s));
  std::vector<double> h(3 * nrhs + 1);
  // eta = ||b - A x||_1 / (||A||_1 ||x||_1 + ||b||_1), worst column; leaves b - A x in R.
  auto eta_now = [&](double* out) -> prrp_status {
    CK(launch_residual(dA_orig, F->lda, n, dB, ldb, nrhs, B0, nrhs, R, ctx->norms, s));
    CK(cudaMemcpyAsync(h.data(), ctx->norms, sizeof(double) * (3 * nrhs + 1),
                       cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double worst = 0.0;
    for (int c = 0; c < nrhs; ++c) {
      const double den = h[3 * nrhs] * h[nrhs + c] + h[2 * nrhs + c];
      worst = std::max(worst, den > 0 ? h[c] / den : (h[c] > 0 ? INFINITY : 0.0));
    }
    *out = worst;
    return PRRP_OK;
  };
  double eta = 0.0;
  if ((ps = eta_now(&eta)) != PRRP_OK) return ps;
  if (info) info->eta0 = eta;

  // One restart cycle of GMRES-based refinement (for low-precision factors whose classic
  // refinement contracts slowly): the correction d of A d = r is found by GMRES on the
  // preconditioned system (LU)^-1 A d = (LU)^-1 r, with the FP32 factors applied as the
  // preconditioner and every other operation in FP64 (products with the original A,
  // classical Gram-Schmidt done twice, Givens rotations of the Hessenberg matrix on the
  // host), nrhs columns side by side.  Every cycle's correction is kept and eta updated: a
  // cycle may raise eta a little and still leave the next ones a better start, so the caller
  // tracks the best iterate in the block after the basis.
  constexpr int m = 30;                     // Krylov vectors per cycle
  constexpr size_t kBest = m + 1;           // block of the krylov buffer holding the best iterate
  int inner = 0;                            // preconditioned GMRES steps (one FP32 solve each)
  auto gmres_cycle = [&]() -> prrp_status {
    constexpr double tol = 1e-10;           // relative decrease of the preconditioned residual
    prrp_status q;
    if ((q = grow(ctx, &ctx->gm_coef, &ctx->gm_coef_cap, (size_t)(m + 1) * nrhs)) != PRRP_OK) return q;
    double* V = ctx->krylov;
    double* W = Y;                          // free in the low-precision path
    double* D = R;                          // R is consumed by the first preconditioner solve
    double* coef = ctx->gm_coef;
    std::vector<double> hv((size_t)(m + 1) * nrhs), h2((size_t)(m + 1) * nrhs), up((size_t)(m + 1) * nrhs);
    auto dots = [&](int nvec, const double* X, double* host) -> prrp_status {
      CK(launch_block_dots(V, nvec, n, nrhs, X, coef, s));
      CK(cudaMemcpyAsync(host, coef, sizeof(double) * nvec * nrhs, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      return PRRP_OK;
    };
    auto precondition = [&](const double* X, double* out) -> prrp_status {   // out = (LU)^-1 X
      prrp_status r = solve_into32(ctx, F, X, nrhs, nrhs, s);
      if (r != PRRP_OK) return r;
      CK(launch_scale_cols(nullptr, ctx->y32, n, nrhs, nullptr, out, s));
      return PRRP_OK;
    };
    if ((q = precondition(R, V)) != PRRP_OK) return q;
    std::vector<double> beta(nrhs);
    if ((q = dots(1, V, hv.data())) != PRRP_OK) return q;
    for (int c = 0; c < nrhs; ++c) {
      beta[c] = std::sqrt(std::max(hv[c], 0.0));
      up[c] = beta[c] > 0.0 ? 1.0 / beta[c] : 0.0;
    }
    CK(cudaMemcpyAsync(coef, up.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
    CK(launch_scale_cols(V, nullptr, n, nrhs, coef, V, s));
    // per column: Hessenberg H ((m + 1) x m, column-major), rotations, right-hand side g
    std::vector<double> H((size_t)nrhs * (m + 1) * m, 0.0), cs((size_t)nrhs * m), sn((size_t)nrhs * m);
    std::vector<double> g((size_t)nrhs * (m + 1), 0.0);
    std::vector<int> kc(nrhs, 0);
    std::vector<char> done(nrhs, 0);
    for (int c = 0; c < nrhs; ++c) { g[(size_t)c * (m + 1)] = beta[c]; done[c] = beta[c] == 0.0; }
    for (int j = 0; j < m; ++j) {
      bool all = true;
      for (int c = 0; c < nrhs; ++c) all = all && done[c];
      if (all) break;
      if ((q = [&]() -> prrp_status {
             CK(launch_matvec(dA_orig, F->lda, n, V + (size_t)j * blk, nrhs, nrhs, D, s));
             return PRRP_OK;
           }()) != PRRP_OK) return q;
      if ((q = precondition(D, W)) != PRRP_OK) return q;
      ++inner;
      // Gram-Schmidt against V_0 .. V_j, twice
      if ((q = dots(j + 1, W, hv.data())) != PRRP_OK) return q;
      CK(launch_block_axpy(V, j + 1, n, nrhs, coef, -1.0, W, s));
      if ((q = dots(j + 1, W, h2.data())) != PRRP_OK) return q;
      CK(launch_block_axpy(V, j + 1, n, nrhs, coef, -1.0, W, s));
      CK(launch_block_dots(W, 1, n, nrhs, W, coef, s));
      std::vector<double> hn(nrhs);
      CK(cudaMemcpyAsync(hn.data(), coef, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (int c = 0; c < nrhs; ++c) {
        const double nrm = std::sqrt(std::max(hn[c], 0.0));
        up[c] = 0.0;
        if (done[c]) continue;
        double* Hc = H.data() + (size_t)c * (m + 1) * m + (size_t)j * (m + 1);   // column j
        for (int i = 0; i <= j; ++i) Hc[i] = hv[(size_t)i * nrhs + c] + h2[(size_t)i * nrhs + c];
        Hc[j + 1] = nrm;
        for (int i = 0; i < j; ++i) {                  // earlier rotations
          const double a = Hc[i], bb = Hc[i + 1];
          Hc[i] = cs[(size_t)c * m + i] * a + sn[(size_t)c * m + i] * bb;
          Hc[i + 1] = -sn[(size_t)c * m + i] * a + cs[(size_t)c * m + i] * bb;
        }
        const double rr = std::hypot(Hc[j], Hc[j + 1]);
        const double cj = rr > 0.0 ? Hc[j] / rr : 1.0, sj = rr > 0.0 ? Hc[j + 1] / rr : 0.0;
        cs[(size_t)c * m + j] = cj;
        sn[(size_t)c * m + j] = sj;
        Hc[j] = rr;
        Hc[j + 1] = 0.0;
        double* gc = g.data() + (size_t)c * (m + 1);
        gc[j + 1] = -sj * gc[j];
        gc[j] = cj * gc[j];
        kc[c] = j + 1;
        if (std::fabs(gc[j + 1]) <= tol * beta[c] || nrm <= 1e-300) done[c] = 1;
        else up[c] = 1.0 / nrm;
      }
      CK(cudaMemcpyAsync(coef, up.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
      CK(launch_scale_cols(W, nullptr, n, nrhs, coef, V + (size_t)(j + 1) * blk, s));
    }
    // y = H^-1 g per column (upper triangular after the rotations), D = sum_i y_i V_i
    int kmax = 0;
    std::fill(hv.begin(), hv.end(), 0.0);
    for (int c = 0; c < nrhs; ++c) {
      const double* Hcol = H.data() + (size_t)c * (m + 1) * m;
      const double* gc = g.data() + (size_t)c * (m + 1);
      for (int i = kc[c] - 1; i >= 0; --i) {
        double acc = gc[i];
        for (int l = i + 1; l < kc[c]; ++l) acc -= Hcol[(size_t)l * (m + 1) + i] * hv[(size_t)l * nrhs + c];
        hv[(size_t)i * nrhs + c] = Hcol[(size_t)i * (m + 1) + i] != 0.0 ? acc / Hcol[(size_t)i * (m + 1) + i] : 0.0;
      }
      kmax = std::max(kmax, kc[c]);
    }
    CK(cudaMemcpyAsync(coef, hv.data(), sizeof(double) * std::max(kmax, 1) * nrhs, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(D, 0, sizeof(double) * blk, s));
    CK(launch_block_axpy(V, kmax, n, nrhs, coef, 1.0, D, s));
    CK(launch_axpy_rows(dB, ldb, D, 1.0, n, nrhs, s));
    return eta_now(&eta);
  };

  int it = 0;
  bool exhausted = false;
  bool gm = false;
  int cycles = 0;
  int stalls = 0;                           // consecutive GMRES cycles without a new best eta
  double best = 0.0;
  auto keep_best = [&]() -> prrp_status {
    CK(launch_copy_rows(dB, ldb, ctx->krylov + kBest * blk, nrhs, n, nrhs, s));
    best = eta;
    return PRRP_OK;
  };
  while (eta > o.refine_target) {
    if (gm) {
      if (cycles == o.refine_max_iter) { exhausted = true; break; }
      if (stalls == 2) break;
      if (cycles == 0) {                     // one allocation for the basis and the best iterate
        if ((ps = grow(ctx, &ctx->krylov, &ctx->krylov_cap, (kBest + 1) * blk)) != PRRP_OK) return ps;
        if ((ps = keep_best()) != PRRP_OK) return ps;
      }
      if ((ps = gmres_cycle()) != PRRP_OK) return ps;
      ++cycles;
      if (eta < best) {
        stalls = 0;
        if ((ps = keep_best()) != PRRP_OK) return ps;
      } else {
        ++stalls;
      }
      continue;
    }
    if (it == o.refine_max_iter) { exhausted = true; break; }
    if (low) {
      if ((ps = solve_into32(ctx, F, R, nrhs, nrhs, s)) != PRRP_OK) return ps;
      CK(launch_axpy_rows32(dB, ldb, ctx->y32, 1.0, n, nrhs, s));
    } else {
      if ((ps = solve_into(ctx, F, R, nrhs, nrhs, Y, s)) != PRRP_OK) return ps;
      CK(launch_axpy_rows(dB, ldb, Y, 1.0, n, nrhs, s));
    }
    double e2 = 0.0;
    if ((ps = eta_now(&e2)) != PRRP_OK) return ps;
    ++it;
    if (low && e2 > eta / 2) {       // slow contraction: continue with GMRES-based refinement
      if (e2 > eta) {                // diverging: back to the previous iterate and its residual
        CK(launch_axpy_rows32(dB, ldb, ctx->y32, -1.0, n, nrhs, s));
        if ((ps = eta_now(&e2)) != PRRP_OK) return ps;
      }
      eta = e2;
      gm = true;
      continue;
    }
    if (e2 > eta / 2) {              // stagnation: keep the better of the last two
      if (e2 > eta) {
        if (low) CK(launch_axpy_rows32(dB, ldb, ctx->y32, -1.0, n, nrhs, s));
        else CK(launch_axpy_rows(dB, ldb, Y, -1.0, n, nrhs, s));
      }
      eta = std::min(eta, e2);
      break;
    }
    eta = e2;
  }
  if (cycles > 0 && eta > best) {           // end on the best GMRES iterate
    CK(launch_copy_rows(ctx->krylov + kBest * blk, nrhs, dB, ldb, n, nrhs, s));
    eta = best;
    exhausted = exhausted && eta > o.refine_target;
  }
  if ((ps = sync_solve(ctx, s)) != PRRP_OK) return ps;
  collect_timing(ctx);
  if (info) { info->iterations = it + inner; info->eta = eta; }
  return exhausted ? PRRP_ERR_NOT_CONVERGED : PRRP_OK;
}

prrp_status prrp_gesv_host(prrp_ctx* ctx, int n, const double* hA, int lda, int nrhs,
                           const double* hB, int ldb, double* hX, const prrp_opts* opts_in,
                           void* stream, prrp_factor_stats* stats, prrp_solve_info* info) {
  if (!ctx || n < 0 || nrhs < 0 || lda < std::max(n, 1) || ldb < std::max(nrhs, 1))
    return PRRP_ERR_INVALID_ARG;
  if (n > 0 && (!hA || (nrhs > 0 && (!hB || !hX)))) return PRRP_ERR_INVALID_ARG;
  prrp_opts o;
  prrp_opts_default(&o);
  if (opts_in) o = *opts_in;
  if (n == 0) return PRRP_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaSetDevice(ctx->device));
  const bool refine = o.refine_max_iter > 0 && nrhs > 0;
  prrp_status ps = grow(ctx, &ctx->hA, &ctx->hA_cap, (size_t)n * n);
  if (ps != PRRP_OK) return ps;
  if (refine && (ps = grow(ctx, &ctx->hA0, &ctx->hA0_cap, (size_t)n * n)) != PRRP_OK) return ps;
  if ((ps = grow(ctx, &ctx->hB, &ctx->hB_cap, (size_t)n * std::max(nrhs, 1))) != PRRP_OK) return ps;
  CK(cudaMemcpy2DAsync(ctx->hA, sizeof(double) * n, hA, sizeof(double) * lda, sizeof(double) * n, n,
                       cudaMemcpyHostToDevice, s));
  if (refine)
    CK(cudaMemcpyAsync(ctx->hA0, ctx->hA, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, s));
  if (nrhs > 0)
    CK(cudaMemcpy2DAsync(ctx->hB, sizeof(double) * nrhs, hB, sizeof(double) * ldb,
                         sizeof(double) * nrhs, n, cudaMemcpyHostToDevice, s));
  prrp_factors* F = nullptr;
  ps = prrp_factor(ctx, n, ctx->hA, n, &o, stream, &F);
  if (stats && F) *stats = F->stats;
  if (ps != PRRP_OK) { prrp_factors_destroy(F); return ps; }
  ps = prrp_solve(ctx, F, refine ? ctx->hA0 : nullptr, nrhs, ctx->hB, std::max(nrhs, 1), &o, stream, info);
  prrp_factors_destroy(F);
  if (ps != PRRP_OK && ps != PRRP_ERR_NOT_CONVERGED) return ps;
  if (nrhs > 0) {
    CK(cudaMemcpy2DAsync(hX, sizeof(double) * ldb, ctx->hB, sizeof(double) * nrhs,
                         sizeof(double) * nrhs, n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  return ps;
}

prrp_status prrp_panel_select(prrp_ctx* ctx, int m, int w, const double* dP, int ldp, double tau,
                              int max_swaps, int* hOrder, double* dL21, int* hSwaps, void* stream) {
  if (!ctx || w < 1 || w > kMaxW || m < w || ldp < w || !dP || !(tau >= 1.0) || max_swaps < 0)
    return PRRP_ERR_INVALID_ARG;
  if (m > w && !dL21) return PRRP_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaSetDevice(ctx->device));
  prrp_status ps = ensure_panel_ws(ctx, m, w, max_swaps);
  if (ps != PRRP_OK) return ps;
  if ((ps = grow_i(ctx, &ctx->order, &ctx->order_cap, m)) != PRRP_OK) return ps;
  CK(cudaMemsetAsync(ctx->st, 0, sizeof(DevState), s));
  {
    Timed t(ctx, s, PRRP_KIND_PANEL);
    ps = enqueue_panel(ctx, dP, ldp, m, w, tau, max_swaps, 0, dL21, w, ctx->order, nullptr, s);
  }
  if (ps != PRRP_OK) return ps;
  DevState h{};
  if ((ps = read_state(ctx, &h, s)) != PRRP_OK) return ps;
  collect_timing(ctx);
  if (hSwaps) *hSwaps = h.panel_swaps;
  if (h.status != 0) return (prrp_status)h.status;
  if (hOrder) CK(cudaMemcpy(hOrder, ctx->order, sizeof(int) * m, cudaMemcpyDeviceToHost));
  return PRRP_OK;
}

prrp_status prrp_schur_update(prrp_ctx* ctx, int m, int n, int k, const double* dL, int ldl,
                              const double* dU, int ldu, double* dC, int ldc, int prec,
                              void* stream) {
  if (!ctx || m < 0 || n < 0 || k < 1 || k > kMaxW || ldl < k || ldu < std::max(n, 1) ||
      ldc < std::max(n, 1))
    return PRRP_ERR_INVALID_ARG;
  if (m > 0 && n > 0 && (!dL || !dU || !dC)) return PRRP_ERR_INVALID_ARG;
  if (prec != PRRP_FP64 && prec != PRRP_TF32 && prec != PRRP_BF16X3 && prec != PRRP_FP64_EMU)
    return PRRP_ERR_UNSUPPORTED;
  if (prec == PRRP_FP64_EMU && k > 64) return PRRP_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaSetDevice(ctx->device));
  CK(cudaMemsetAsync(ctx->st, 0, sizeof(DevState), s));
  if (prec == PRRP_FP64) {
    Timed t(ctx, s, PRRP_KIND_UPDATE, 2LL * m * n * k);
    CK(launch_gemm_fp64(m, n, k, dL, ldl, dU, ldu, dC, ldc, ctx->st, 0, ctx->num_sms, s));
  } else {
    prrp_status ps = grow(ctx, &ctx->tcws, &ctx->tcws_cap, tc_workspace_bytes(prec, m, n, k));
    if (ps != PRRP_OK) return ps;
    Timed t(ctx, s, PRRP_KIND_UPDATE, 2LL * m * n * k);
    CK(launch_tc_update(prec, m, n, k, dL, ldl, dU, ldu, dC, ldc, ctx->st, 0, ctx->tcws, s));
  }
  DevState h{};
  prrp_status ps = read_state(ctx, &h, s);
  if (ps != PRRP_OK) return ps;
  collect_timing(ctx);
  return (prrp_status)h.status;
}

// ---------------------------------------------------------------- batched solves
namespace {

struct BatchPlan {
  int nmax, b, tmp_rows, grid;
  size_t wsW_elems, per_cta_bytes;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Per-CTA workspace: W (nmax^2 T), Tmp rows (tmp_rows x nmax T), V (5 nmax doubles),
// I (3 nmax ints).
size_t batch_cta_bytes(int nmax, int tmp_rows, bool fp64) {
  const size_t tb = fp64 ? 8 : 4;
  return align256((size_t)nmax * nmax * tb) + align256((size_t)tmp_rows * nmax * tb) +
         align256((size_t)5 * nmax * 8) + align256((size_t)3 * nmax * 4);
}

int batch_max_ctas_per_sm(int nmax, int b) {
  int per = 0;
  // every instantiation is capped at 128 registers a thread (two CTAs of 256 threads per
  // SM) and holds at most 26 KB of static shared memory beside the dynamic panel space
  const size_t smem = batch_smem_bytes(nmax, b);
  if (smem > 200 * 1024) return 0;
  per = (int)std::min<size_t>(2, (228 * 1024) / (smem + 26 * 1024 + 1024));
  return std::max(per, 1);
}

// Enqueue one batched launch (counter reset + kernel) over metadata already on the device.
prrp_status enqueue_batch(prrp_ctx* ctx, bool fp64, int count, int nmax, int b, int tmp_rows,
                          int grid, int rb, const prrp_opts& o, const int* d_order, const int* d_n,
                          const double* const* d_A, const int* d_lda, const int* d_nrhs,
                          double* const* d_B, const int* d_ldb, int* const* d_perm, int* d_status, int* d_iters,
                          double* d_eta0, double* d_eta, unsigned* d_counter, cudaStream_t s) {
  const size_t per = batch_cta_bytes(nmax, tmp_rows, fp64);
  BatchLaunch L{};
  L.count = count; L.order = d_order; L.n = d_n; L.A = d_A; L.lda = d_lda; L.nrhs = d_nrhs;
  L.B = d_B; L.ldb = d_ldb; L.perm_out = d_perm; L.b = b; L.tau = o.tau; L.max_swaps = o.max_swaps;
  L.refine_max_iter = o.refine_max_iter; L.refine_target = o.refine_target; L.nmax = nmax;
  const size_t tb = fp64 ? 8 : 4;
  unsigned char* base = ctx->bws;
  L.wsW = base;
  base += align256((size_t)grid * nmax * nmax * tb);
  L.wsT = base;
  base += align256((size_t)grid * tmp_rows * nmax * tb);
  L.tmp_rows = tmp_rows;
  L.wsV = reinterpret_cast<double*>(base);
  base += align256((size_t)grid * 5 * nmax * 8);
  L.wsI = reinterpret_cast<int*>(base);
  (void)per;
  L.status = d_status; L.iters = d_iters; L.eta0 = d_eta0; L.eta = d_eta; L.counter = d_counter;
  CK(cudaMemsetAsync(d_counter, 0, sizeof(unsigned), s));
  CK(launch_batch(fp64 ? 1 : 0, grid, rb, L, s));
  return PRRP_OK;
}

size_t batch_ws_bytes(int grid, int nmax, int tmp_rows, bool fp64) {
  const size_t tb = fp64 ? 8 : 4;
  return align256((size_t)grid * nmax * nmax * tb) + align256((size_t)grid * tmp_rows * nmax * tb) +
         align256((size_t)grid * 5 * nmax * 8) + align256((size_t)grid * 3 * nmax * 4) + 1024;
}

}  // namespace

// Batched launch shape: CTAs per SM (1 .. maxper) x the update's register tile (1 or 2 rows
// of L21 per warp pass), timed on a synthetic sample of full-bucket systems.  The choice
// depends only on the device, precision, b and size bucket, so it is kept per process (and
// per context, for the lock-free lookup): lanes of a server and later servers reuse it.
// Tuning holds a process-wide lock, so two contexts never time their candidates against
// each other.
static std::mutex g_tune_mu;
static std::map<std::pair<int, long long>, int> g_tuned;   // (device, key) -> 4 * per + rb

static prrp_status batch_tune_run(prrp_ctx* ctx, bool fp64, int b, int bucket, const prrp_opts& o, int maxper,
                                  cudaStream_t s, int* out) {
  prrp_status ps = PRRP_OK;
  const int ns = 128 * bucket > 1024 ? 1024 : 128 * bucket;
  const int sample = std::min(2 * ctx->num_sms, 256);
  // owners: every return below (CK included) frees the sample and the events
  struct DevMem { void* p = nullptr; ~DevMem() { if (p) cudaFree(p); } } mA, mB;
  struct Ev { cudaEvent_t e = nullptr; ~Ev() { if (e) cudaEventDestroy(e); } } e0, e1;
  CK(cudaMalloc(&mA.p, sizeof(double) * (size_t)sample * ns * ns));
  CK(cudaMalloc(&mB.p, sizeof(double) * (size_t)sample * ns));
  CK(cudaEventCreate(&e0.e));
  CK(cudaEventCreate(&e1.e));
  double* tA = static_cast<double*>(mA.p);
  double* tB = static_cast<double*>(mB.p);
  std::vector<int> hn(sample, ns), hl(sample, ns), hr(sample, 1), hord(sample);
  std::iota(hord.begin(), hord.end(), 0);
  std::vector<const double*> ha(sample);
  std::vector<double*> hb(sample);
  for (int i = 0; i < sample; ++i) { ha[i] = tA + (size_t)i * ns * ns; hb[i] = tB + (size_t)i * ns; }
  int best = 4 * 1 + 1;
  float best_ms = 1e30f;
  const int nrb = fp64 ? 1 : 2;                         // FP64 keeps one row per pass
  for (int cand = 0; cand < nrb * maxper && ps == PRRP_OK; ++cand) {
    const int per = 1 + cand / nrb, rb = 1 + cand % nrb;
    const int grid = per * ctx->num_sms;
    ps = grow(ctx, &ctx->bws, &ctx->bws_cap, batch_ws_bytes(grid, ns, std::min(ns, 2 * (b + o.max_swaps) + 2), fp64));
    if (ps != PRRP_OK) break;
    const size_t mb = align256(sizeof(int) * sample * 6) + align256(sizeof(void*) * sample * 2);
    ps = grow(ctx, &ctx->bmeta, &ctx->bmeta_cap, mb + 256);
    if (ps != PRRP_OK) break;
    ps = grow(ctx, &ctx->bout, &ctx->bout_cap, align256(sizeof(int) * 2 * sample) + align256(sizeof(double) * 2 * sample) + 256);
    if (ps != PRRP_OK) break;
    int* mi = reinterpret_cast<int*>(ctx->bmeta);
    CK(cudaMemcpyAsync(mi, hord.data(), sizeof(int) * sample, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(mi + sample, hn.data(), sizeof(int) * sample, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(mi + 2 * sample, hl.data(), sizeof(int) * sample, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(mi + 3 * sample, hr.data(), sizeof(int) * sample, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(mi + 4 * sample, hr.data(), sizeof(int) * sample, cudaMemcpyHostToDevice, s));
    const double** pa = reinterpret_cast<const double**>(ctx->bmeta + align256(sizeof(int) * sample * 6));
    double** pb = reinterpret_cast<double**>(ctx->bmeta + align256(sizeof(int) * sample * 6) +
                                             sizeof(void*) * sample);
    CK(cudaMemcpyAsync(pa, ha.data(), sizeof(void*) * sample, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(pb, hb.data(), sizeof(void*) * sample, cudaMemcpyHostToDevice, s));
    int* d_status = reinterpret_cast<int*>(ctx->bout);
    int* d_iters = d_status + sample;
    double* d_e0 = reinterpret_cast<double*>(ctx->bout + align256(sizeof(int) * 2 * sample));
    double* d_e = d_e0 + sample;
    unsigned* d_counter = reinterpret_cast<unsigned*>(mi + 5 * sample);
    float ms = 0.f;
    for (int rep = 0; rep < 2 && ps == PRRP_OK; ++rep) {   // first run warms up
      CK(launch_batch_fill(tA, ns, sample, tB, s));
      CK(cudaEventRecord(e0.e, s));
      ps = enqueue_batch(ctx, fp64, sample, ns, b, std::min(ns, 2 * (b + o.max_swaps) + 2), grid, rb, o, mi,
                         mi + sample, pa, mi + 2 * sample, mi + 3 * sample, pb, mi + 4 * sample,
                         nullptr, d_status, d_iters, d_e0, d_e, d_counter, s);
      CK(cudaEventRecord(e1.e, s));
      CK(cudaEventSynchronize(e1.e));
      CK(cudaEventElapsedTime(&ms, e0.e, e1.e));
    }
    if (ps != PRRP_OK) break;
    if (ms < best_ms) { best_ms = ms; best = 4 * per + rb; }
  }
  if (ps != PRRP_OK) return ps;
  *out = best;
  return PRRP_OK;
}

static prrp_status batch_shape(prrp_ctx* ctx, bool fp64, int b, int bucket, const prrp_opts& o, int maxper,
                               cudaStream_t s, int* out) {
  const long long tkey = ((long long)fp64 << 40) | ((long long)b << 20) | bucket;
  auto it = ctx->batch_tuned.find(tkey);
  if (it != ctx->batch_tuned.end()) {
    *out = 4 * std::min(it->second / 4, maxper) + it->second % 4;
    return PRRP_OK;
  }
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto g = g_tuned.find({ctx->device, tkey});
  if (g == g_tuned.end()) {
    int best = 0;
    prrp_status ps = batch_tune_run(ctx, fp64, b, bucket, o, maxper, s, &best);
    if (ps != PRRP_OK) return ps;
    g = g_tuned.emplace(std::make_pair(ctx->device, tkey), best).first;
  }
  ctx->batch_tuned[tkey] = g->second;
  // a shape tuned on full-bucket systems never asks for more CTAs per SM than fit, but
  // one tuned first on smaller systems of the bucket may: clamp to this batch's limit
  *out = 4 * std::min(g->second / 4, maxper) + g->second % 4;
  return PRRP_OK;
}

prrp_status prrp_batch_tune(prrp_ctx* ctx, int nmax, const prrp_opts* opts_in, void* stream) {
  if (!ctx || nmax < 1) return PRRP_ERR_INVALID_ARG;
  if (nmax > 1024) return PRRP_ERR_UNSUPPORTED;
  prrp_opts o;
  prrp_opts_default(&o);
  o.b = 16;
  o.prec = PRRP_FP32;
  if (opts_in) o = *opts_in;
  prrp_status ps = check_opts(&o);
  if (ps != PRRP_OK) return ps;
  if (o.prec != PRRP_FP32 && o.prec != PRRP_FP64) return PRRP_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaSetDevice(ctx->device));
  for (int bucket = 1; bucket <= (nmax + 127) / 128; ++bucket) {
    const int nb = 128 * bucket;
    const int b = std::min({o.b, batch_max_width(), nb});
    const int maxper = batch_max_ctas_per_sm(nb, b);
    if (maxper == 0) return PRRP_ERR_UNSUPPORTED;
    CK(prepare_batch(nb, b));
    int shape = 0;
    if ((ps = batch_shape(ctx, o.prec == PRRP_FP64, b, bucket, o, maxper, s, &shape)) != PRRP_OK) return ps;
  }
  return PRRP_OK;
}

prrp_status prrp_batch_solve(prrp_ctx* ctx, int count, const int* n, const double* const* dA,
                             const int* lda, const int* nrhs, double* const* dB, const int* ldb,
                             int* const* dPerm, const prrp_opts* opts_in, void* stream,
                             prrp_status* per_system, prrp_solve_info* info) {
  if (!ctx || count < 0 || (count > 0 && (!n || !dA || !lda || !nrhs || !dB || !ldb)))
    return PRRP_ERR_INVALID_ARG;
  prrp_opts o;
  prrp_opts_default(&o);
  o.b = 16;
  o.prec = PRRP_FP32;
  if (opts_in) o = *opts_in;
  prrp_status ps = check_opts(&o);
  if (ps != PRRP_OK) return ps;
  if (o.prec != PRRP_FP32 && o.prec != PRRP_FP64) return PRRP_ERR_UNSUPPORTED;
  if (count == 0) return PRRP_OK;
  int nmax = 1;
  for (int i = 0; i < count; ++i) {
    if (n[i] < 1 || lda[i] < n[i] || nrhs[i] < 0 || ldb[i] < std::max(nrhs[i], 1) || !dA[i] ||
        (nrhs[i] > 0 && !dB[i]))
      return PRRP_ERR_INVALID_ARG;
    nmax = std::max(nmax, n[i]);
  }
  if (nmax > 1024) return PRRP_ERR_UNSUPPORTED;
  const int b = std::min({o.b, batch_max_width(), nmax});
  const bool fp64 = o.prec == PRRP_FP64;
  const int tmp_rows = std::min(nmax, 2 * (b + o.max_swaps) + 2);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaSetDevice(ctx->device));
  const int maxper = batch_max_ctas_per_sm(nmax, b);
  if (maxper == 0) return PRRP_ERR_UNSUPPORTED;
  CK(prepare_batch(std::max(nmax, 128 * ((nmax + 127) / 128)), b));

  // ---- the launch shape for this (precision, b, size bucket): tuned once per process
  int shape = 0;
  if ((ps = batch_shape(ctx, fp64, b, (nmax + 127) / 128, o, maxper, s, &shape)) != PRRP_OK) return ps;
  const int grid = (shape / 4) * ctx->num_sms, rb = shape % 4;

  // ---- metadata: largest systems first, so the tail of the work list is short
  std::vector<int> ord(count);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return n[x] > n[y]; });
  const size_t ints = align256(sizeof(int) * ((size_t)count * 6 + 1));
  const size_t ptrs = align256(sizeof(void*) * (size_t)count * 3);
  if ((ps = grow(ctx, &ctx->bmeta, &ctx->bmeta_cap, ints + ptrs + 256)) != PRRP_OK) return ps;
  if ((ps = grow(ctx, &ctx->bws, &ctx->bws_cap, batch_ws_bytes(grid, nmax, tmp_rows, fp64))) != PRRP_OK) return ps;
  const size_t outb = align256(sizeof(int) * 2 * (size_t)count) + align256(sizeof(double) * 2 * (size_t)count);
  if ((ps = grow(ctx, &ctx->bout, &ctx->bout_cap, outb + 256)) != PRRP_OK) return ps;
  std::vector<unsigned char> host(ints + ptrs, 0);
  int* hi = reinterpret_cast<int*>(host.data());
  std::copy(ord.begin(), ord.end(), hi);
  std::copy(n, n + count, hi + count);
  std::copy(lda, lda + count, hi + 2 * count);
  std::copy(nrhs, nrhs + count, hi + 3 * count);
  std::copy(ldb, ldb + count, hi + 4 * count);
  std::memcpy(host.data() + ints, dA, sizeof(void*) * count);
  std::memcpy(host.data() + ints + sizeof(void*) * count, dB, sizeof(void*) * count);
  if (dPerm) std::memcpy(host.data() + ints + 2 * sizeof(void*) * count, dPerm, sizeof(void*) * count);
  CK(cudaMemcpyAsync(ctx->bmeta, host.data(), host.size(), cudaMemcpyHostToDevice, s));
  int* mi = reinterpret_cast<int*>(ctx->bmeta);
  const double* const* pa = reinterpret_cast<const double* const*>(ctx->bmeta + ints);
  double* const* pb = reinterpret_cast<double* const*>(ctx->bmeta + ints + sizeof(void*) * count);
  int* const* pp = reinterpret_cast<int* const*>(ctx->bmeta + ints + 2 * sizeof(void*) * count);
  int* d_status = reinterpret_cast<int*>(ctx->bout);
  int* d_iters = d_status + count;
  double* d_e0 = reinterpret_cast<double*>(ctx->bout + align256(sizeof(int) * 2 * (size_t)count));
  double* d_e = d_e0 + count;
  unsigned* d_counter = reinterpret_cast<unsigned*>(mi + 5 * count);

  // ---- the launch sequence, replayed as a captured CUDA graph while its shape is unchanged
  long long tau_bits, tgt_bits;
  std::memcpy(&tau_bits, &o.tau, 8);
  std::memcpy(&tgt_bits, &o.refine_target, 8);
  const std::vector<long long> sig = {count, nmax, grid, rb, fp64, b, tmp_rows, tau_bits, o.max_swaps, dPerm != nullptr,
                                      o.refine_max_iter, tgt_bits, (long long)(uintptr_t)ctx->bws,
                                      (long long)(uintptr_t)ctx->bmeta, (long long)(uintptr_t)ctx->bout};
  if (ctx->bgraph.sig != sig || !ctx->bgraph.exec) {
    if (ctx->bgraph.exec) { cudaGraphExecDestroy(ctx->bgraph.exec); ctx->bgraph.exec = nullptr; }
    if (!ctx->capture_stream) CK(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
    ps = enqueue_batch(ctx, fp64, count, nmax, b, tmp_rows, grid, rb, o, mi, mi + count, pa, mi + 2 * count,
                       mi + 3 * count, pb, mi + 4 * count, dPerm ? pp : nullptr, d_status, d_iters, d_e0,
                       d_e, d_counter, ctx->capture_stream);
    cudaError_t ce = cudaStreamEndCapture(ctx->capture_stream, &g);
    if (ps != PRRP_OK) { if (g) cudaGraphDestroy(g); return ps; }
    if (ce != cudaSuccess) return cuda_fail(ctx, ce, "batch graph capture");
    ce = cudaGraphInstantiate(&ctx->bgraph.exec, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return cuda_fail(ctx, ce, "batch graph instantiate");
    ctx->bgraph.sig = sig;
  }
  {
    Timed t(ctx, s, PRRP_KIND_BATCH);
    CK(cudaGraphLaunch(ctx->bgraph.exec, s));
  }
  std::vector<int> hs(2 * (size_t)count);
  std::vector<double> he(2 * (size_t)count);
  CK(cudaMemcpyAsync(hs.data(), d_status, sizeof(int) * 2 * count, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(he.data(), d_e0, sizeof(double) * 2 * count, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  collect_timing(ctx);
  prrp_status first = PRRP_OK;
  for (int i = 0; i < count; ++i) {
    const prrp_status si = static_cast<prrp_status>(hs[i]);
    if (per_system) per_system[i] = si;
    if (info) { info[i].iterations = hs[count + i]; info[i].eta0 = he[i]; info[i].eta = he[count + i]; }
    if (si != PRRP_OK && first == PRRP_OK) first = si;
  }
  return first;
}

prrp_status prrp_ctx_device(const prrp_ctx* ctx, int* device) {
  if (!ctx || !device) return PRRP_ERR_INVALID_ARG;
  *device = ctx->device;
  return PRRP_OK;
}

prrp_status prrp_ctx_set_timing(prrp_ctx* ctx, int enable) {
  if (!ctx || enable < 0 || enable > 2) return PRRP_ERR_INVALID_ARG;
  ctx->timing = enable != 0;
  ctx->timeline.clear();
  if (enable == 2) {
    CK(cudaSetDevice(ctx->device));
    if (!ctx->tl_base) CK(cudaEventCreate(&ctx->tl_base));
    CK(cudaEventRecord(ctx->tl_base, 0));
    CK(cudaEventSynchronize(ctx->tl_base));
  } else if (ctx->tl_base) {
    cudaEventDestroy(ctx->tl_base);
    ctx->tl_base = nullptr;
  }
  return PRRP_OK;
}

prrp_status prrp_ctx_set_panel_mode(prrp_ctx* ctx, int cluster_max_rows) {
  if (!ctx || cluster_max_rows < 0 || cluster_max_rows > 4096) return PRRP_ERR_INVALID_ARG;
  ctx->panel_cluster_rows = cluster_max_rows;
  return PRRP_OK;
}

prrp_status prrp_ctx_set_sm_split(prrp_ctx* ctx, int panel_ctas, int block_ctas) {
  if (!ctx || panel_ctas < 0 || block_ctas < 0 || panel_ctas > ctx->num_sms || block_ctas > ctx->num_sms)
    return PRRP_ERR_INVALID_ARG;
  if (panel_ctas < ctx->num_sms && panel_ctas + block_ctas > ctx->num_sms - 8) return PRRP_ERR_INVALID_ARG;
  ctx->split_panel = panel_ctas;
  ctx->split_blk = block_ctas;
  return PRRP_OK;
}

prrp_status prrp_ctx_set_update_block(prrp_ctx* ctx, int nb) {
  if (!ctx || nb < 0 || nb > kAggMaxNB) return PRRP_ERR_INVALID_ARG;
  ctx->agg_nb = nb;
  return PRRP_OK;
}

prrp_status prrp_ctx_set_solve_mode(prrp_ctx* ctx, int mode) {
  if (!ctx || mode < 0 || mode > 1) return PRRP_ERR_INVALID_ARG;
  ctx->solve_mode = mode;
  return PRRP_OK;
}

prrp_status prrp_ctx_timeline(prrp_ctx* ctx, int cap, int* kinds, double* t0_ms, double* t1_ms, int* count) {
  if (!ctx || cap < 0 || !count || (cap > 0 && (!kinds || !t0_ms || !t1_ms))) return PRRP_ERR_INVALID_ARG;
  const int n = static_cast<int>(std::min<size_t>(ctx->timeline.size(), static_cast<size_t>(cap)));
  for (int i = 0; i < n; ++i) {
    kinds[i] = ctx->timeline[i].kind;
    t0_ms[i] = ctx->timeline[i].t0;
    t1_ms[i] = ctx->timeline[i].t1;
  }
  *count = static_cast<int>(ctx->timeline.size());
  return PRRP_OK;
}

prrp_status prrp_ctx_kernel_stats(prrp_ctx* ctx, double* ms, long long* launches,
                                  long long* flops, int reset) {
  if (!ctx) return PRRP_ERR_INVALID_ARG;
  for (int k = 0; k < PRRP_KIND_COUNT; ++k) {
    if (ms) ms[k] = ctx->kind_ms[k];
    if (launches) launches[k] = ctx->kind_launches[k];
    if (flops) flops[k] = ctx->kind_flops[k];
    if (reset) { ctx->kind_ms[k] = 0; ctx->kind_launches[k] = 0; ctx->kind_flops[k] = 0; }
  }
  return PRRP_OK;
}

prrp_status prrp_selftest_wait(prrp_ctx* ctx, unsigned spin_limit, void* stream) {
  if (!ctx) return PRRP_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaSetDevice(ctx->device));
  CK(cudaMemsetAsync(ctx->st, 0, sizeof(DevState), s));
  CK(cudaMemcpyAsync(&ctx->st->spin_limit, &spin_limit, sizeof(unsigned), cudaMemcpyHostToDevice, s));
  CK(launch_wait_selftest(ctx->st, s));
  DevState h{};
  prrp_status ps = read_state(ctx, &h, s);
  if (ps != PRRP_OK) return ps;
  CK(cudaMemsetAsync(ctx->st, 0, sizeof(DevState), s));
  CK(cudaStreamSynchronize(s));
  return (prrp_status)h.status;
}

prrp_status prrp_selftest_chain_wait(prrp_ctx* ctx, unsigned spin_limit, void* stream) {
  if (!ctx) return PRRP_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaSetDevice(ctx->device));
  const size_t words = trsv_counter_words(128);
  prrp_status ps;
  if (ctx->tcount_cap < words) {
    if ((ps = grow(ctx, &ctx->tcount, &ctx->tcount_cap, words)) != PRRP_OK) return ps;
  }
  if ((ps = grow(ctx, &ctx->zbuf, &ctx->zbuf_cap, (kChainSelftestFloats + 1) / 2)) != PRRP_OK) return ps;
  CK(cudaMemsetAsync(ctx->st, 0, sizeof(DevState), s));
  CK(cudaMemcpyAsync(&ctx->st->spin_limit, &spin_limit, sizeof(unsigned), cudaMemcpyHostToDevice, s));
  CK(launch_trsv_chain_selftest(reinterpret_cast<float*>(ctx->zbuf), ctx->tcount, ctx->st, s));
  ps = sync_solve(ctx, s);                  // reports and clears the recorded site
  CK(cudaMemsetAsync(ctx->st, 0, sizeof(DevState), s));
  CK(cudaStreamSynchronize(s));
  return ps;
}

}  // extern "C"
