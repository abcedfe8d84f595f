// Continuous-batching request server over cPINN / XPINN models (see the
// serving section of xpinn.h).
//
// Threads: one dispatcher admits submitted requests in arrival order while
// the in-flight device-memory footprint fits the budget; one worker per
// model owns a CUDA stream and serves every admitted request of its model,
// stitching runs of evaluation requests with the same copy and derivative
// order into one routed evaluation (Eq. FSol) and running training steps in
// arrival order.  Workers of different models run concurrently, so their
// kernels overlap on the GPU.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "xpinn.h"

namespace xp {
int ctx_out_total(xpinn_handle h);
int ctx_n_sub(xpinn_handle h);
int ctx_n_copies(xpinn_handle h);
int ctx_device(xpinn_handle h);
void set_last_error(const char* msg);
}  // namespace xp

using Clock = std::chrono::steady_clock;

namespace {

struct Req {
  uint64_t ticket;
  xpinn_request r;
  size_t bytes;
  Clock::time_point t_submit, t_admit;
};

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

int n_comp(int order) { return order == 0 ? 1 : (order == 1 ? 3 : 5); }

}  // namespace

struct xpinn_server {
  std::vector<xpinn_handle> models;
  size_t budget = 0, in_flight = 0;
  std::mutex mu;
  std::condition_variable cv_disp;
  std::vector<std::condition_variable> cv_work;
  std::deque<Req> pending;
  std::vector<std::deque<Req>> admitted;
  std::unordered_map<uint64_t, xpinn_result> done;
  std::unordered_set<uint64_t> live;
  uint64_t next = 1;
  bool stop = false;
  std::thread dispatcher;
  std::vector<std::thread> workers;

  explicit xpinn_server(size_t n) : cv_work(n), admitted(n) {}
};

namespace {

// Device bytes an evaluation of n points needs in the routed path: points,
// membership and routing arrays, up to one entry per point for each box it
// lies in (one in the interior), entry outputs and the stitched output.
size_t eval_bytes(xpinn_handle h, int64_t n, int order) {
  const size_t row = (size_t)xp::ctx_out_total(h) * n_comp(order);
  return (size_t)n * (8 + 4 + 16 + 16 + 2 * (8 + 4 + 4 * row) + 4 * row);
}

void finish(xpinn_server* s, Req& q, int status, int batch) {
  const auto now = Clock::now();
  xpinn_result r;
  r.status = status;
  r.queue_ms = ms_between(q.t_submit, q.t_admit);
  r.latency_ms = ms_between(q.t_submit, now);
  r.batch = batch;
  memset(r.error, 0, sizeof r.error);
  if (status != XPINN_OK) strncpy(r.error, xpinn_last_error(), sizeof r.error - 1);
  std::lock_guard<std::mutex> lk(s->mu);
  s->in_flight -= q.bytes;
  s->live.erase(q.ticket);
  s->done[q.ticket] = r;
  s->cv_disp.notify_all();
}

void dispatcher_loop(xpinn_server* s) {
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv_disp.wait(lk, [&] {
      return s->stop || (!s->pending.empty() && s->in_flight + s->pending.front().bytes <= s->budget);
    });
    if (s->stop && s->pending.empty()) return;
    while (!s->pending.empty() && s->in_flight + s->pending.front().bytes <= s->budget) {
      Req q = s->pending.front();
      s->pending.pop_front();
      q.t_admit = Clock::now();
      s->in_flight += q.bytes;
      const int m = q.r.model;
      s->admitted[m].push_back(q);
      s->cv_work[m].notify_one();
    }
    if (s->stop && s->pending.empty()) return;
  }
}

void worker_loop(xpinn_server* s, int m) {
  xpinn_handle h = s->models[m];
  cudaSetDevice(xp::ctx_device(h));
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  std::vector<float> xy, out;
  for (;;) {
    std::vector<Req> batch;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work[m].wait(lk, [&] { return s->stop || !s->admitted[m].empty(); });
      if (s->admitted[m].empty()) {
        if (s->stop) break;
        continue;
      }
      batch.assign(s->admitted[m].begin(), s->admitted[m].end());
      s->admitted[m].clear();
    }
    size_t i = 0;
    while (i < batch.size()) {
      Req& q = batch[i];
      if (q.r.kind == XPINN_REQ_STEP) {
        const int rc = xpinn_step(h, q.r.n_steps, q.r.losses, st);
        finish(s, q, rc, 1);
        ++i;
        continue;
      }
      // a run of evaluations with the same copy and order: one launch
      size_t j = i;
      int64_t n = 0;
      while (j < batch.size() && batch[j].r.kind == XPINN_REQ_EVAL && batch[j].r.copy == q.r.copy &&
             batch[j].r.order == q.r.order) {
        n += batch[j].r.n;
        ++j;
      }
      const int row = xp::ctx_out_total(h) * n_comp(q.r.order);
      xy.resize(2 * (size_t)n);
      out.resize((size_t)n * row);
      int64_t off = 0;
      for (size_t k = i; k < j; ++k) {
        memcpy(xy.data() + 2 * off, batch[k].r.xy, sizeof(float) * 2 * batch[k].r.n);
        off += batch[k].r.n;
      }
      const int rc = n ? xpinn_eval(h, q.r.copy, xy.data(), n, q.r.order, out.data(), st) : XPINN_OK;
      off = 0;
      for (size_t k = i; k < j; ++k) {
        if (rc == XPINN_OK)
          memcpy(batch[k].r.out, out.data() + off * row, sizeof(float) * row * batch[k].r.n);
        off += batch[k].r.n;
        finish(s, batch[k], rc, (int)(j - i));
      }
      i = j;
    }
  }
  cudaStreamDestroy(st);
}

int fail(int code, const char* msg) {
  xp::set_last_error(msg);
  return code;
}

}  // namespace

extern "C" {

int xpinn_server_create(const xpinn_handle* models, int32_t n_models, size_t hbm_budget,
                        xpinn_server** out) {
  if (!models || n_models < 1 || !out || hbm_budget == 0) return fail(XPINN_ERR_INVALID, "bad arguments");
  for (int m = 0; m < n_models; ++m)
    if (!models[m]) return fail(XPINN_ERR_INVALID, "NULL model handle");
  try {
    auto* s = new xpinn_server((size_t)n_models);
    s->models.assign(models, models + n_models);
    s->budget = hbm_budget;
    s->dispatcher = std::thread(dispatcher_loop, s);
    for (int m = 0; m < n_models; ++m) s->workers.emplace_back(worker_loop, s, m);
    *out = s;
  } catch (...) {
    return fail(XPINN_ERR_INVALID, "could not start the server threads");
  }
  xp::set_last_error("");
  return XPINN_OK;
}

int xpinn_server_submit(xpinn_server* s, const xpinn_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket) return fail(XPINN_ERR_INVALID, "bad arguments");
  if (req->model < 0 || req->model >= (int)s->models.size()) return fail(XPINN_ERR_INVALID, "bad model");
  xpinn_handle h = s->models[req->model];
  size_t bytes = 0;
  if (req->kind == XPINN_REQ_EVAL) {
    if (req->n < 0 || (req->n > 0 && (!req->xy || !req->out)) || req->order < 0 || req->order > 2 ||
        req->copy < 0 || req->copy >= xp::ctx_n_copies(h))
      return fail(XPINN_ERR_INVALID, "bad evaluation request");
    bytes = eval_bytes(h, req->n, req->order);
  } else if (req->kind == XPINN_REQ_STEP) {
    if (req->n_steps < 0) return fail(XPINN_ERR_INVALID, "bad step request");
  } else {
    return fail(XPINN_ERR_INVALID, "unknown request kind");
  }
  if (bytes > s->budget) return fail(XPINN_ERR_OOM, "request larger than the server's memory budget");
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return fail(XPINN_ERR_INVALID, "server is stopping");
  Req q;
  q.ticket = s->next++;
  q.r = *req;
  q.bytes = bytes;
  q.t_submit = Clock::now();
  q.t_admit = q.t_submit;
  s->pending.push_back(q);
  s->live.insert(q.ticket);
  s->cv_disp.notify_all();
  *ticket = q.ticket;
  return XPINN_OK;
}

int xpinn_server_poll(xpinn_server* s, uint64_t ticket, xpinn_result* res) {
  if (!s || !res) return fail(XPINN_ERR_INVALID, "bad arguments");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->done.find(ticket);
  if (it != s->done.end()) {
    *res = it->second;
    s->done.erase(it);
    return XPINN_OK;
  }
  if (s->live.count(ticket)) return XPINN_PENDING;
  return fail(XPINN_ERR_INVALID, "unknown ticket");
}

int xpinn_server_destroy(xpinn_server* s) {
  if (!s) return XPINN_OK;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_disp.wait(lk, [&] { return s->live.empty(); });
    s->stop = true;
    s->cv_disp.notify_all();
    for (auto& c : s->cv_work) c.notify_all();
  }
  s->dispatcher.join();
  for (auto& t : s->workers) t.join();
  delete s;
  return XPINN_OK;
}

}  // extern "C"
