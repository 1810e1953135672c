// C ABI of libprrp.so: argument checks, device workspace, and the host-side loop of
// Algorithm 1 that enqueues one panel's kernels after another on the caller's stream.
// Every pivot decision stays on the device; the host reads the device state word once,
// after the last panel.
#include <cuda_runtime.h>

#include <algorithm>
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

struct prrp_ctx {
  int device = 0;
  int num_sms = 0;
  size_t smem_optin = 0;
  DevState* st = nullptr;       // device
  double* xval = nullptr;       // panel exchange records
  int2* xkey = nullptr;
  double* xvec = nullptr;
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
  std::string last_error;
  // optional per-kernel-class timing with CUDA events on the launching stream
  bool timing = false;
  struct Rec { cudaEvent_t a, b; int kind; };
  std::vector<Rec> recs;
  size_t nrec = 0;
  double kind_ms[PRRP_KIND_COUNT] = {};
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
  if (o->prec < PRRP_FP64 || o->prec > PRRP_FP32) return PRRP_ERR_INVALID_ARG;
  if (o->refine_max_iter < 0) return PRRP_ERR_INVALID_ARG;
  return PRRP_OK;
}

// Cooperative grid size for an m-row panel: <= one CTA per SM, >= 32 rows per CTA.
prrp_status panel_grid(prrp_ctx* ctx, int m, int w, int* G, int* rpc) {
  int g = std::max(1, std::min(ctx->num_sms, (m + 31) / 32));
  int r = (m + g - 1) / g;
  if (panel_smem_for(w, r) > ctx->smem_optin) return PRRP_ERR_UNSUPPORTED;
  *G = g;
  *rpc = r;
  return PRRP_OK;
}

prrp_status ensure_panel_ws(prrp_ctx* ctx, int n, int w, int max_swaps) {
  prrp_status s;
  if (ctx->xcap < 2 * ctx->num_sms) {
    const int G = 2 * ctx->num_sms;
    size_t c1 = 0, c2 = 0, c3 = 0;
    if (ctx->xval) { cudaFree(ctx->xval); cudaFree(ctx->xkey); cudaFree(ctx->xvec); }
    ctx->xval = nullptr; ctx->xkey = nullptr; ctx->xvec = nullptr;
    if ((s = grow(ctx, &ctx->xval, &c1, 2 * (size_t)G)) != PRRP_OK) return s;
    if ((s = grow(ctx, &ctx->xkey, &c2, 2 * (size_t)G)) != PRRP_OK) return s;
    if ((s = grow(ctx, &ctx->xvec, &c3, 2 * (size_t)G * kMaxW)) != PRRP_OK) return s;
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
                          int* pairs, cudaStream_t s) {
  int G = 0, rpc = 0;
  prrp_status ps = panel_grid(ctx, m, w, &G, &rpc);
  if (ps != PRRP_OK) return ps;
  CK(cudaMemsetAsync(&ctx->st->barrier, 0, 2 * sizeof(unsigned), s));
  PanelParams p{};
  p.P = P; p.ldp = ldp; p.m = m; p.w = w; p.tau = tau; p.max_swaps = max_swaps;
  p.col_offset = col_offset; p.L21 = L21; p.ldl = ldl; p.order = order; p.pairs = pairs;
  p.st = ctx->st; p.xval = ctx->xval; p.xkey = ctx->xkey; p.xvec = ctx->xvec; p.rows_per_cta = rpc;
  cudaError_t e = launch_panel(p, G, s);
  if (e == cudaErrorCooperativeLaunchTooLarge) return PRRP_ERR_UNSUPPORTED;
  if (e != cudaSuccess) return cuda_fail(ctx, e, "panel launch");
  return PRRP_OK;
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
  void* ptrs[] = {ctx->st, ctx->xval, ctx->xkey, ctx->xvec, ctx->pairs, ctx->ipiv, ctx->order,
                  ctx->l21, ctx->solve_ws, ctx->norms, ctx->hA, ctx->hA0, ctx->hB, ctx->tcws};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete ctx;
  return PRRP_OK;
}

prrp_status prrp_factor(prrp_ctx* ctx, int n, double* dA, int lda, const prrp_opts* opts_in,
                        void* stream, prrp_factors** F) {
  if (!ctx || !F) return PRRP_ERR_INVALID_ARG;
  *F = nullptr;
  prrp_opts o;
  prrp_opts_default(&o);
  if (opts_in) o = *opts_in;
  if (n < 0 || lda < std::max(n, 1) || (n > 0 && !dA)) return PRRP_ERR_INVALID_ARG;
  prrp_status ps = check_opts(&o);
  if (ps != PRRP_OK) return ps;
  if (o.prec == PRRP_FP32) return PRRP_ERR_UNSUPPORTED;
  if (n > 65536) return PRRP_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaSetDevice(ctx->device));

  prrp_factors* f = new (std::nothrow) prrp_factors();
  if (!f) return PRRP_ERR_OOM;
  f->ctx = ctx; f->n = n; f->dA = dA; f->lda = lda; f->opts = o;
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
  for (int k0 = 0; k0 < n; k0 += b) {
    const int w = std::min(b, n - k0), m = n - k0;
    double* Akk = dA + (long long)k0 * lda + k0;
    {
      Timed t(ctx, s, PRRP_KIND_PANEL, 3LL * m * w * w);
      ps = enqueue_panel(ctx, Akk, lda, m, w, o.tau, o.max_swaps, k0, ctx->l21, w, nullptr,
                         ctx->pairs, s);
    }
    if (ps != PRRP_OK) return fail(ps);
    {
      Timed t(ctx, s, PRRP_KIND_PERMUTE);
      e = launch_permute(dA, lda, n, k0, ctx->pairs, max_pairs, f->perm, ctx->st, s);
    }
    if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "permute"));
    if (m > w) {
      Timed t(ctx, s, PRRP_KIND_UPDATE, 2LL * (m - w) * (n - k0 - w) * w);
      if (o.prec == PRRP_FP64)
        e = launch_gemm_fp64(m - w, n - k0 - w, w, ctx->l21, w, Akk + w, lda,
                             Akk + (long long)w * lda + w, lda, ctx->st, 1, ctx->num_sms, s);
      else
        e = launch_tc_update(o.prec, m - w, n - k0 - w, w, ctx->l21, w, Akk + w, lda,
                             Akk + (long long)w * lda + w, lda, ctx->st, 1, ctx->tcws, s);
      if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "schur update"));
    }
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
    if (m > w) {
      Timed t(ctx, s, PRRP_KIND_LFIX, 1LL * (m - w) * w * w);
      e = launch_lfix(dA, lda, n, k0, w, ctx->l21, w, ctx->ipiv, ctx->st, s);
    }
    if (e != cudaSuccess) return fail(cuda_fail(ctx, e, "lfix"));
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

static prrp_status solve_into(prrp_ctx* ctx, const prrp_factors* F, const double* B, long long ldb,
                              int nrhs, double* Y, cudaStream_t s) {
  cudaError_t e;
  const int nb = (F->n + 63) / 64;
  Timed t(ctx, s, PRRP_KIND_SOLVE, 2LL * F->n * F->n * nrhs);
  ctx->kind_launches[PRRP_KIND_SOLVE] += 2LL * nb;   // gather + 2 nb substitution steps
  if ((e = launch_gather_rows(B, ldb, F->perm, F->n, nrhs, Y, s)) != cudaSuccess) return cuda_fail(ctx, e, "gather");
  if ((e = launch_trsv_lower_unit(F->dA, F->lda, F->n, Y, nrhs, s)) != cudaSuccess) return cuda_fail(ctx, e, "trsv L");
  if ((e = launch_trsv_upper(F->dA, F->lda, F->n, Y, nrhs, s)) != cudaSuccess) return cuda_fail(ctx, e, "trsv U");
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
  if (refine) CK(launch_copy_rows(dB, ldb, B0, nrhs, n, nrhs, s));
  if ((ps = solve_into(ctx, F, dB, ldb, nrhs, Y, s)) != PRRP_OK) return ps;
  {
    Timed t(ctx, s, PRRP_KIND_SOLVE);
    CK(launch_copy_rows(Y, nrhs, dB, ldb, n, nrhs, s));
  }
  if (!refine) {
    CK(cudaStreamSynchronize(s));
    collect_timing(ctx);
    return PRRP_OK;
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
  int it = 0;
  bool exhausted = false;
  while (eta > o.refine_target) {
    if (it == o.refine_max_iter) { exhausted = true; break; }
    if ((ps = solve_into(ctx, F, R, nrhs, nrhs, Y, s)) != PRRP_OK) return ps;
    CK(launch_axpy_rows(dB, ldb, Y, 1.0, n, nrhs, s));
    double e2 = 0.0;
    if ((ps = eta_now(&e2)) != PRRP_OK) return ps;
    ++it;
    if (e2 > eta / 2) {              // stagnation: keep the better of the last two
      if (e2 > eta) CK(launch_axpy_rows(dB, ldb, Y, -1.0, n, nrhs, s));
      eta = std::min(eta, e2);
      break;
    }
    eta = e2;
  }
  CK(cudaStreamSynchronize(s));
  collect_timing(ctx);
  if (info) { info->iterations = it; info->eta = eta; }
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
  ps = enqueue_panel(ctx, dP, ldp, m, w, tau, max_swaps, 0, dL21, w, ctx->order, nullptr, s);
  if (ps != PRRP_OK) return ps;
  DevState h{};
  if ((ps = read_state(ctx, &h, s)) != PRRP_OK) return ps;
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
  if (prec != PRRP_FP64 && prec != PRRP_TF32 && prec != PRRP_BF16X3) return PRRP_ERR_UNSUPPORTED;
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

prrp_status prrp_ctx_set_timing(prrp_ctx* ctx, int enable) {
  if (!ctx) return PRRP_ERR_INVALID_ARG;
  ctx->timing = enable != 0;
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

}  // extern "C"
