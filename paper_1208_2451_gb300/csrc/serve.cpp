// Serving loop for LU_PRRP solves: continuous batching of incoming requests on one GPU.
//
// Requests (n x n system, 1..many right-hand sides, host buffers) are queued by
// prrp_server_submit and admitted against an HBM budget.  `lanes` worker threads each own
// a prrp_ctx and a CUDA stream; whenever a lane is idle it takes the next unit of work:
//   * the queued requests with n <= 512 that fit the remaining budget, up to 512 of them,
//     solved together by one prrp_batch_solve launch (FP32 working copy, FP64 pivot
//     selection and refinement, or the FP64 form), or
//   * one request with n > 512: prrp_factor (Schur update in the configured precision,
//     FP64 pivoting) into device memory that holds its factors until prrp_solve has
//     refined its right-hand sides in FP64 against the device copy of A.
// Requests that arrive while every lane is busy wait in the queue and join the next unit a
// lane forms, so work keeps flowing onto the device as lanes and memory free up, and the
// lanes' launches overlap on the GPU.  Each system's arithmetic does not depend on which
// unit it lands in, so a result is bit-identical alone and in a mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "prrp.h"

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kSmallMax = 512;    // largest n sent to the batched kernel (one CTA per system)
constexpr int kUnitMax = 512;     // most requests in one batched unit

struct Item {
  prrp_request req;
  size_t bytes = 0;
  Clock::time_point t_submit, t_start, t_done;
  bool done = false;
  prrp_result res{};
};

}  // namespace

struct prrp_server {
  int device = 0;
  size_t budget = 0;
  prrp_opts opts{};
  int nlanes = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Item> items;
  size_t in_use = 0, peak_in_use = 0;
  int busy_lanes = 0, peak_busy_lanes = 0;
  bool stop = false;
  uint64_t next_id = 1;
  uint64_t submitted = 0, completed = 0, rejected = 0, units = 0;
  std::vector<double> latencies_us;
  Clock::time_point t_first_submit, t_last_done;
  bool any_submit = false;
  std::vector<std::thread> lanes;
  std::atomic<int> lane_errors{0};
};

namespace {

size_t request_bytes(int n, int nrhs) {
  // device A (+ FP64 copy of A for the refinement residual, + FP32 copy of the factors for
  // the correction solves), right-hand sides, factor workspace (multipliers, solve scratch)
  const size_t nn = static_cast<size_t>(n) * n;
  return 20 * nn + 40 * static_cast<size_t>(n) * std::max(nrhs, 1) + 1024 * static_cast<size_t>(n) + 4096;
}

double us_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::micro>(b - a).count();
}

// Device buffers of one unit, from the stream-ordered pool.
struct DevBufs {
  std::vector<void*> ptrs;
  cudaStream_t s;
  void* get(size_t bytes) {
    void* p = nullptr;
    if (cudaMallocAsync(&p, std::max<size_t>(bytes, 16), s) != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return p;
  }
  void release() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
    ptrs.clear();
  }
};

// One attempt at a batched unit; returns false when an allocation failed (nothing of the
// unit has been written then) so the caller can retry once memory frees up.
bool try_small_unit(prrp_server* S, prrp_ctx* ctx, cudaStream_t s, std::vector<Item*>& unit) {
  const int cnt = static_cast<int>(unit.size());
  DevBufs db{{}, s};
  std::vector<int> n(cnt), lda(cnt), nrhs(cnt), ldb(cnt);
  std::vector<const double*> dA(cnt);
  std::vector<double*> dB(cnt);
  bool ok = true;
  cudaError_t copy = cudaSuccess;      // first failed copy of the unit (reported per request)
  auto track = [&](cudaError_t e) { if (copy == cudaSuccess) copy = e; };
  for (int i = 0; i < cnt && ok; ++i) {
    const prrp_request& r = unit[i]->req;
    n[i] = r.n; lda[i] = r.n; nrhs[i] = r.nrhs; ldb[i] = std::max(r.nrhs, 1);
    double* a = static_cast<double*>(db.get(sizeof(double) * r.n * r.n));
    double* b = static_cast<double*>(db.get(sizeof(double) * r.n * std::max(r.nrhs, 1)));
    if (!a || !b) { ok = false; break; }
    track(cudaMemcpy2DAsync(a, sizeof(double) * r.n, r.hA, sizeof(double) * r.lda, sizeof(double) * r.n, r.n,
                            cudaMemcpyHostToDevice, s));
    if (r.nrhs > 0)
      track(cudaMemcpy2DAsync(b, sizeof(double) * r.nrhs, r.hB, sizeof(double) * r.ldb, sizeof(double) * r.nrhs,
                              r.n, cudaMemcpyHostToDevice, s));
    dA[i] = a;
    dB[i] = b;
  }
  std::vector<prrp_status> st(cnt, PRRP_ERR_OOM);
  std::vector<prrp_solve_info> info(cnt);
  if (ok && copy == cudaSuccess) {
    prrp_opts o = S->opts;
    if (o.prec != PRRP_FP64) o.prec = PRRP_FP32;
    o.b = std::min(o.b, 16);
    const prrp_status rc = prrp_batch_solve(ctx, cnt, n.data(), dA.data(), lda.data(), nrhs.data(), dB.data(),
                                            ldb.data(), nullptr, &o, s, st.data(), info.data());
    if (rc == PRRP_ERR_OOM || rc == PRRP_ERR_CUDA) {
      std::fprintf(stderr, "prrp_server: batched unit of %d: %s (%s)\n", cnt, prrp_status_string(rc),
                   prrp_ctx_last_error(ctx));
      if (rc == PRRP_ERR_OOM) ok = false;
    }
    for (int i = 0; i < cnt && ok; ++i) {
      const prrp_request& r = unit[i]->req;
      if (st[i] == PRRP_OK && r.nrhs > 0)
        track(cudaMemcpy2DAsync(r.hX, sizeof(double) * r.ldx, dB[i], sizeof(double) * r.nrhs,
                                sizeof(double) * r.nrhs, r.n, cudaMemcpyDeviceToHost, s));
    }
  }
  db.release();
  track(cudaStreamSynchronize(s));
  if (!ok) return false;
  for (int i = 0; i < cnt; ++i) {
    unit[i]->res.status = copy == cudaSuccess ? st[i] : PRRP_ERR_CUDA;
    unit[i]->res.eta = info[i].eta;
    unit[i]->res.iterations = info[i].iterations;
  }
  return true;
}

// Allocation failures are retried with a short back-off (other lanes may be releasing
// memory) for up to ~2 s before the unit's requests fail with PRRP_ERR_OOM.
void run_small_unit(prrp_server* S, prrp_ctx* ctx, cudaStream_t s, std::vector<Item*>& unit) {
  for (int attempt = 0; attempt < 400; ++attempt) {
    if (try_small_unit(S, ctx, s, unit)) return;
    cudaGetLastError();
    std::this_thread::sleep_for(std::chrono::milliseconds(5));
  }
  for (Item* it : unit) it->res.status = PRRP_ERR_OOM;
}

bool try_big_item(prrp_server* S, prrp_ctx* ctx, cudaStream_t s, Item* it) {
  const prrp_request& r = it->req;
  DevBufs db{{}, s};
  const size_t nn = static_cast<size_t>(r.n) * r.n;
  double* a = static_cast<double*>(db.get(sizeof(double) * nn));
  double* a0 = static_cast<double*>(db.get(sizeof(double) * nn));
  double* b = static_cast<double*>(db.get(sizeof(double) * r.n * std::max(r.nrhs, 1)));
  prrp_status st = PRRP_ERR_OOM;
  prrp_solve_info info{0, -1.0, -1.0};
  cudaError_t copy = cudaSuccess;      // first failed copy (the request then fails with PRRP_ERR_CUDA)
  auto track = [&](cudaError_t e) { if (copy == cudaSuccess) copy = e; };
  if (a && a0 && b) {
    track(cudaMemcpy2DAsync(a0, sizeof(double) * r.n, r.hA, sizeof(double) * r.lda, sizeof(double) * r.n, r.n,
                            cudaMemcpyHostToDevice, s));
    track(cudaMemcpyAsync(a, a0, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
    if (r.nrhs > 0)
      track(cudaMemcpy2DAsync(b, sizeof(double) * r.nrhs, r.hB, sizeof(double) * r.ldb, sizeof(double) * r.nrhs,
                              r.n, cudaMemcpyHostToDevice, s));
    prrp_opts o = S->opts;
    if (o.prec == PRRP_FP32) o.prec = PRRP_BF16X3;
    prrp_factors* F = nullptr;
    st = copy == cudaSuccess ? prrp_factor(ctx, r.n, a, r.n, &o, s, &F) : PRRP_ERR_CUDA;
    if (st == PRRP_ERR_OOM || st == PRRP_ERR_CUDA)
      std::fprintf(stderr, "prrp_server: n=%d factor: %s (%s)\n", r.n, prrp_status_string(st),
                   prrp_ctx_last_error(ctx));
    if (st == PRRP_OK && r.nrhs > 0) {
      st = prrp_solve(ctx, F, a0, r.nrhs, b, r.nrhs, &o, s, &info);
      if (st == PRRP_OK || st == PRRP_ERR_NOT_CONVERGED)
        track(cudaMemcpy2DAsync(r.hX, sizeof(double) * r.ldx, b, sizeof(double) * r.nrhs, sizeof(double) * r.nrhs,
                                r.n, cudaMemcpyDeviceToHost, s));
    }
    prrp_factors_destroy(F);
  }
  db.release();
  track(cudaStreamSynchronize(s));
  if (st == PRRP_ERR_OOM) return false;
  if (copy != cudaSuccess && st == PRRP_OK) st = PRRP_ERR_CUDA;
  it->res.status = st;
  it->res.eta = info.eta;
  it->res.iterations = info.iterations;
  return true;
}

void run_big_item(prrp_server* S, prrp_ctx* ctx, cudaStream_t s, Item* it) {
  for (int attempt = 0; attempt < 400; ++attempt) {
    if (try_big_item(S, ctx, s, it)) return;
    cudaGetLastError();
    std::this_thread::sleep_for(std::chrono::milliseconds(5));
  }
  it->res.status = PRRP_ERR_OOM;
}

void lane_main(prrp_server* S) {
  cudaSetDevice(S->device);
  prrp_ctx* ctx = nullptr;
  if (prrp_create(&ctx, S->device) != PRRP_OK) { S->lane_errors++; return; }
  // lanes factor side by side: panels up to 2048 rows as co-scheduled clusters, which do
  // not wait for the other lanes' panels (taller ones are faster as a grid)
  prrp_ctx_set_panel_mode(ctx, 2048);
  cudaStream_t s;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  for (;;) {
    std::vector<Item*> unit;
    size_t unit_bytes = 0;
    bool big = false;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (;;) {
        if (S->stop && S->queue.empty()) break;
        // admission: the first queued request that fits the remaining budget decides the
        // unit's kind; small ones behind it that also fit join a batched unit
        for (auto qi = S->queue.begin(); qi != S->queue.end();) {
          Item& it = S->items[*qi];
          const bool is_big = it.req.n > kSmallMax;
          if (S->in_use + unit_bytes + it.bytes > S->budget || (!unit.empty() && (is_big || big))) {
            ++qi;
            continue;
          }
          unit.push_back(&it);
          unit_bytes += it.bytes;
          big = is_big;
          qi = S->queue.erase(qi);
          if (big || static_cast<int>(unit.size()) >= kUnitMax) break;
        }
        if (!unit.empty()) break;
        S->cv_work.wait(lk);
      }
      if (unit.empty()) break;
      S->in_use += unit_bytes;
      S->peak_in_use = std::max(S->peak_in_use, S->in_use);
      S->busy_lanes++;
      S->peak_busy_lanes = std::max(S->peak_busy_lanes, S->busy_lanes);
      S->units++;
      const auto now = Clock::now();
      for (Item* it : unit) it->t_start = now;
    }
    if (big) run_big_item(S, ctx, s, unit[0]);
    else run_small_unit(S, ctx, s, unit);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      const auto now = Clock::now();
      for (Item* it : unit) {
        it->t_done = now;
        it->done = true;
        it->res.latency_us = us_between(it->t_submit, now);
        it->res.queue_us = us_between(it->t_submit, it->t_start);
        S->latencies_us.push_back(it->res.latency_us);
        S->completed++;
      }
      S->t_last_done = now;
      S->in_use -= unit_bytes;
      S->busy_lanes--;
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
  cudaStreamDestroy(s);
  prrp_destroy(ctx);
}

}  // namespace

extern "C" {

prrp_status prrp_server_create(prrp_ctx* ctx, size_t hbm_budget_bytes, const prrp_opts* opts, int lanes,
                               prrp_server** out) {
  if (!ctx || !out || hbm_budget_bytes == 0 || lanes < 1 || lanes > 16) return PRRP_ERR_INVALID_ARG;
  *out = nullptr;
  prrp_server* S = new (std::nothrow) prrp_server();
  if (!S) return PRRP_ERR_OOM;
  int dev = 0;
  if (prrp_ctx_device(ctx, &dev) != PRRP_OK) { delete S; return PRRP_ERR_INVALID_ARG; }
  S->device = dev;
  S->budget = hbm_budget_bytes;
  prrp_opts_default(&S->opts);
  S->opts.prec = PRRP_FP32;
  if (opts) S->opts = *opts;
  S->nlanes = lanes;
  // the batched units' launch shapes are tuned here, before any request waits on them
  prrp_opts bo = S->opts;
  if (bo.prec != PRRP_FP64) bo.prec = PRRP_FP32;
  bo.b = std::min(bo.b, 16);
  const prrp_status ts = prrp_batch_tune(ctx, kSmallMax, &bo, nullptr);
  if (ts != PRRP_OK) { delete S; return ts; }
  for (int i = 0; i < lanes; ++i) S->lanes.emplace_back(lane_main, S);
  *out = S;
  return PRRP_OK;
}

prrp_status prrp_server_submit(prrp_server* S, const prrp_request* r, uint64_t* ticket) {
  if (!S || !r || !ticket || r->n < 1 || r->nrhs < 0 || !r->hA || r->lda < r->n ||
      (r->nrhs > 0 && (!r->hB || !r->hX || r->ldb < r->nrhs || r->ldx < r->nrhs)))
    return PRRP_ERR_INVALID_ARG;
  const size_t bytes = request_bytes(r->n, r->nrhs);
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) return PRRP_ERR_INVALID_ARG;
  if (bytes > S->budget) {
    S->rejected++;
    return PRRP_ERR_BUSY;
  }
  const uint64_t id = S->next_id++;
  Item& it = S->items[id];
  it.req = *r;
  it.bytes = bytes;
  it.t_submit = Clock::now();
  if (!S->any_submit) { S->t_first_submit = it.t_submit; S->any_submit = true; }
  S->queue.push_back(id);
  S->submitted++;
  *ticket = id;
  S->cv_work.notify_one();
  return PRRP_OK;
}

prrp_status prrp_server_wait(prrp_server* S, uint64_t ticket, int64_t timeout_us, prrp_result* out) {
  if (!S) return PRRP_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  auto found = S->items.find(ticket);
  if (found == S->items.end()) return PRRP_ERR_INVALID_ARG;
  auto pred = [&] { return found->second.done; };
  if (timeout_us < 0) S->cv_done.wait(lk, pred);
  else if (!S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), pred)) return PRRP_ERR_TIMEOUT;
  if (out) *out = found->second.res;
  S->items.erase(found);
  return PRRP_OK;
}

prrp_status prrp_server_stats(prrp_server* S, prrp_serve_stats* st) {
  if (!S || !st) return PRRP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  std::memset(st, 0, sizeof(*st));
  st->submitted = S->submitted;
  st->completed = S->completed;
  st->rejected = S->rejected;
  st->units = S->units;
  st->peak_bytes_in_use = S->peak_in_use;
  st->peak_busy_lanes = S->peak_busy_lanes;
  std::vector<double> v = S->latencies_us;
  if (!v.empty()) {
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) { return v[std::min(v.size() - 1, static_cast<size_t>(p * (v.size() - 1) + 0.5))]; };
    st->p50_us = pct(0.50);
    st->p99_us = pct(0.99);
    double sum = 0;
    for (double x : v) sum += x;
    st->mean_us = sum / v.size();
    const double span = us_between(S->t_first_submit, S->t_last_done);
    st->solves_per_s = span > 0 ? 1e6 * v.size() / span : 0.0;
  }
  return PRRP_OK;
}

prrp_status prrp_server_destroy(prrp_server* S) {
  if (!S) return PRRP_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->lanes) t.join();
  const bool lane_failed = S->lane_errors.load() != 0;
  delete S;
  return lane_failed ? PRRP_ERR_CUDA : PRRP_OK;
}

}  // extern "C"
