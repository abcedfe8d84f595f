// Continuous-batching request server over cPINN / XPINN models (see the
// serving section of xpinn.h).
//
// One scheduler thread turns the queue of submitted requests into ticks.  A
// tick takes requests in arrival order while their footprint fits the free
// part of two rings allocated once at creation: device memory (hbm_budget
// bytes) for every request's workspace and device-side inputs and outputs,
// and page-locked host memory for staging its host inputs and outputs.  No
// request allocates.  Within a tick:
//   - evaluation queries of the same model, copy and derivative order become
//     one routed evaluation (Eq. FSol) over all their points, planned on the
//     device (xpinn_eval_ws): one grouped launch for all of them;
//   - training requests on a subdomain subset with their own points run on a
//     private fork of the model (xpinn_fork_step);
//   - whole-model training steps (xpinn_step) train the model in place, in
//     arrival order with that model's other requests.
// The work of one model is queued on one stream (the handle's kernels share
// its scratch), models on different streams, so ticks and models overlap on
// the GPU.  Host inputs are copied into the staging ring on the scheduler
// thread and uploaded asynchronously; outputs come back through it, and are
// copied to the caller's buffers once the tick's events have completed, so
// enqueuing never waits for the GPU.  Ticks complete in order, so both rings
// free their regions first in, first out.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
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
int ctx_sub_params(xpinn_handle h, int q);
int* ctx_err_word(xpinn_handle h);
int fork_sizes(xpinn_handle h, const xpinn_fork_desc* d, size_t* ws_bytes, size_t* table_bytes);
int fork_enqueue(xpinn_handle h, const xpinn_fork_desc* d, void* workspace, size_t ws_bytes, float* dev_losses,
                 float* dev_params, char* pinned, cudaStream_t s);
void set_last_error(const char* msg);
}  // namespace xp

using Clock = std::chrono::steady_clock;

namespace {

constexpr int N_STREAMS = 4;              // models map to streams round-robin
constexpr int MAX_TICK_REQUESTS = 512;    // requests per tick (latency bound)
constexpr int MAX_INFLIGHT_TICKS = 8;

size_t al256(size_t x) { return (x + 255) / 256 * 256; }
int n_comp(int order) { return order == 0 ? 1 : (order == 1 ? 3 : 5); }

// A FIFO ring over [0, cap): regions are taken in order and released in the
// same order (ticks complete in order), so the space in use is one span or
// two (wrapped).
struct Ring {
  size_t cap = 0;
  std::deque<std::pair<size_t, size_t>> used;   // (offset, bytes), oldest first
  bool take(size_t need, size_t& off) {
    if (need == 0) need = 256;
    if (need > cap) return false;
    if (used.empty()) {
      off = 0;
    } else {
      const size_t head = used.back().first + used.back().second, tail = used.front().first;
      const bool wrapped = used.back().first < tail;
      if (!wrapped) {
        if (head + need <= cap) off = head;
        else if (need <= tail) off = 0;
        else return false;
      } else {
        if (head + need <= tail) off = head;
        else return false;
      }
    }
    used.emplace_back(off, need);
    return true;
  }
  void release_oldest() { used.pop_front(); }
};

struct Req {
  uint64_t ticket;
  xpinn_request r;
  size_t dev_bytes = 0, host_bytes = 0;   // footprint in the two rings
  size_t fork_ws = 0, fork_tables = 0;    // forks: workspace and staged table bytes
  int64_t fork_pts = 0;
  int64_t fork_params = 0;
  Clock::time_point t_submit, t_admit;
  int status = XPINN_OK;
  char error[160] = {0};
  int batch = 1;
};

// Slices of a tick's regions given to one unit of work.
struct Unit {
  int kind = XPINN_REQ_EVAL;
  int model = 0, copy = 0, order = 0;
  std::vector<size_t> reqs;   // indices into the tick's requests
  int64_t n = 0;              // eval: points of all requests
  size_t dev_off = 0, host_off = 0;
};

struct Tick {
  std::vector<Req> reqs;
  std::vector<Unit> units;
  size_t dev_off = 0, dev_bytes = 0, host_off = 0, host_bytes = 0;
  std::vector<int> models;                // models with work in the tick
  size_t status_off = 0;                  // host ring: one int per model (device error words)
  cudaEvent_t ev[N_STREAMS] = {};
  bool used_stream[N_STREAMS] = {};
};

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct xpinn_server {
  std::vector<xpinn_handle> models;
  size_t budget = 0;
  char* dev = nullptr;            // device ring memory
  char* host = nullptr;           // page-locked staging ring memory
  Ring dring, hring;
  cudaStream_t streams[N_STREAMS] = {};
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req> pending;
  std::deque<Tick> inflight;
  std::unordered_map<uint64_t, xpinn_result> done;
  std::unordered_set<uint64_t> live;
  uint64_t next = 1;
  bool stop = false;
  std::thread sched;
  int device = 0;
};

namespace {

// Device and host bytes of one request, fixed at submission.
int footprint(xpinn_server* s, Req& q, char* msg, size_t msg_len) {
  const xpinn_request& r = q.r;
  xpinn_handle h = s->models[r.model];
  if (r.kind == XPINN_REQ_EVAL) {
    size_t ws = 0;
    if (xpinn_eval_workspace_size(h, r.copy, r.n, r.order, &ws) != XPINN_OK) {
      snprintf(msg, msg_len, "%s", xpinn_last_error());
      return XPINN_ERR_INVALID;
    }
    const size_t io = al256(8 * (size_t)r.n) + al256(4 * (size_t)r.n * xp::ctx_out_total(h) * n_comp(r.order));
    q.dev_bytes = al256(ws) + io;
    q.host_bytes = io;
  } else if (r.kind == XPINN_REQ_FORK) {
    xpinn_fork_desc d{r.n_sel, r.sel, r.n_pts, r.xy, r.f, r.n_steps};
    const int rc = xp::fork_sizes(h, &d, &q.fork_ws, &q.fork_tables);
    if (rc != XPINN_OK) {
      snprintf(msg, msg_len, "%s", xpinn_last_error());
      return rc;
    }
    for (int i = 0; i < r.n_sel; ++i) {
      q.fork_pts += r.n_pts[i];
      q.fork_params += xp::ctx_sub_params(h, r.sel[i]);
    }
    const size_t io = al256(8 * (size_t)q.fork_pts) + al256(4 * (size_t)q.fork_pts) +
                      al256(4 * (size_t)r.n_steps * r.n_sel * XPINN_N_TERMS) + al256(4 * (size_t)q.fork_params);
    q.dev_bytes = al256(q.fork_ws) + io;
    q.host_bytes = io + al256(q.fork_tables);
  } else {
    const size_t io = al256(4 * (size_t)r.n_steps * xp::ctx_n_sub(h) * XPINN_N_TERMS);
    q.dev_bytes = io;   // the step itself runs on the model's resident buffers
    q.host_bytes = io;
  }
  return XPINN_OK;
}

void fail_req(Req& q, int code, const char* msg) {
  q.status = code;
  snprintf(q.error, sizeof q.error, "%s", msg);
}

// Queues one tick's work; records per-request errors of the enqueue itself.
void enqueue_tick(xpinn_server* s, Tick& t) {
  char* dbase = s->dev + t.dev_off;
  char* hbase = s->host + t.host_off;
  auto stream_of = [&](int model) { return model % N_STREAMS; };
  for (Unit& u : t.units) {
    xpinn_handle h = s->models[u.model];
    const int si = stream_of(u.model);
    cudaStream_t st = s->streams[si];
    t.used_stream[si] = true;
    char* d = dbase + u.dev_off;
    char* hp = hbase + u.host_off;
    if (u.kind == XPINN_REQ_EVAL) {
      const int row = xp::ctx_out_total(h) * n_comp(u.order);
      size_t ws = 0;
      xpinn_eval_workspace_size(h, u.copy, u.n, u.order, &ws);
      float2* dxy = reinterpret_cast<float2*>(d + al256(ws));
      float* dout = reinterpret_cast<float*>(d + al256(ws) + al256(8 * (size_t)u.n));
      float* hxy = reinterpret_cast<float*>(hp);
      int64_t off = 0;
      for (size_t k : u.reqs) {
        const xpinn_request& r = t.reqs[k].r;
        memcpy(hxy + 2 * off, r.xy, sizeof(float) * 2 * r.n);
        off += r.n;
      }
      int rc = cudaMemcpyAsync(dxy, hxy, 8 * (size_t)u.n, cudaMemcpyHostToDevice, st) == cudaSuccess
                   ? XPINN_OK : XPINN_ERR_CUDA;
      if (rc == XPINN_OK)
        rc = xpinn_eval_ws(h, u.copy, reinterpret_cast<float*>(dxy), u.n, u.order, dout, d, ws, st);
      if (rc == XPINN_OK &&
          cudaMemcpyAsync(hp + al256(8 * (size_t)u.n), dout, 4 * (size_t)u.n * row, cudaMemcpyDeviceToHost, st) !=
              cudaSuccess)
        rc = XPINN_ERR_CUDA;
      if (rc != XPINN_OK)
        for (size_t k : u.reqs) fail_req(t.reqs[k], rc, xpinn_last_error());
    } else if (u.kind == XPINN_REQ_FORK) {
      Req& q = t.reqs[u.reqs[0]];
      const xpinn_request& r = q.r;
      const size_t np = (size_t)q.fork_pts;
      float* dxy = reinterpret_cast<float*>(d + al256(q.fork_ws));
      float* df = reinterpret_cast<float*>(reinterpret_cast<char*>(dxy) + al256(8 * np));
      float* dl = reinterpret_cast<float*>(reinterpret_cast<char*>(df) + al256(4 * np));
      const size_t lbytes = 4 * (size_t)r.n_steps * r.n_sel * XPINN_N_TERMS;
      float* dp = reinterpret_cast<float*>(reinterpret_cast<char*>(dl) + al256(lbytes));
      char* hxy = hp;
      char* hf = hxy + al256(8 * np);
      char* hl = hf + al256(4 * np);
      char* hpar = hl + al256(lbytes);
      char* htab = hpar + al256(4 * (size_t)q.fork_params);
      memcpy(hxy, r.xy, 8 * np);
      if (r.f) memcpy(hf, r.f, 4 * np);
      int rc = XPINN_OK;
      if (np && (cudaMemcpyAsync(dxy, hxy, 8 * np, cudaMemcpyHostToDevice, st) != cudaSuccess ||
                 (r.f && cudaMemcpyAsync(df, hf, 4 * np, cudaMemcpyHostToDevice, st) != cudaSuccess)))
        rc = XPINN_ERR_CUDA;
      xpinn_fork_desc fd{r.n_sel, r.sel, r.n_pts, dxy, r.f ? df : nullptr, r.n_steps};
      if (rc == XPINN_OK) rc = xp::fork_enqueue(h, &fd, d, q.fork_ws, dl, dp, htab, st);
      if (rc == XPINN_OK && ((lbytes && cudaMemcpyAsync(hl, dl, lbytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
                             cudaMemcpyAsync(hpar, dp, 4 * (size_t)q.fork_params, cudaMemcpyDeviceToHost, st) !=
                                 cudaSuccess))
        rc = XPINN_ERR_CUDA;
      if (rc != XPINN_OK) fail_req(q, rc, xpinn_last_error());
    } else {
      Req& q = t.reqs[u.reqs[0]];
      const xpinn_request& r = q.r;
      const size_t lbytes = 4 * (size_t)r.n_steps * xp::ctx_n_sub(h) * XPINN_N_TERMS;
      float* dl = reinterpret_cast<float*>(d);
      int rc = xpinn_step(h, r.n_steps, lbytes ? dl : nullptr, st);
      if (rc == XPINN_OK && lbytes && cudaMemcpyAsync(hp, dl, lbytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = XPINN_ERR_CUDA;
      if (rc != XPINN_OK) fail_req(q, rc, xpinn_last_error());
    }
  }
  // each model's device error word: read into the staging ring, then cleared
  int* status = reinterpret_cast<int*>(hbase + t.status_off);
  for (size_t i = 0; i < t.models.size(); ++i) {
    xpinn_handle h = s->models[t.models[i]];
    cudaStream_t st = s->streams[stream_of(t.models[i])];
    status[i] = 0;
    cudaMemcpyAsync(status + i, xp::ctx_err_word(h), sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaMemsetAsync(xp::ctx_err_word(h), 0, sizeof(int), st);
  }
  for (int i = 0; i < N_STREAMS; ++i)
    if (t.used_stream[i]) {
      cudaEventCreateWithFlags(&t.ev[i], cudaEventDisableTiming);
      cudaEventRecord(t.ev[i], s->streams[i]);
    }
}

bool tick_done(const Tick& t) {
  for (int i = 0; i < N_STREAMS; ++i)
    if (t.ev[i] && cudaEventQuery(t.ev[i]) == cudaErrorNotReady) return false;
  return true;
}

// Copies a completed tick's outputs to the callers' buffers; returns results.
void complete_tick(xpinn_server* s, Tick& t, std::vector<std::pair<uint64_t, xpinn_result>>& out) {
  for (int i = 0; i < N_STREAMS; ++i)
    if (t.ev[i]) {
      if (cudaEventSynchronize(t.ev[i]) != cudaSuccess)
        for (Req& q : t.reqs)
          if (q.status == XPINN_OK) fail_req(q, XPINN_ERR_CUDA, "CUDA error in the request's work");
      cudaEventDestroy(t.ev[i]);
    }
  char* hbase = s->host + t.host_off;
  const int* status = reinterpret_cast<const int*>(hbase + t.status_off);
  const auto now = Clock::now();
  for (Unit& u : t.units) {
    xpinn_handle h = s->models[u.model];
    const char* hp = hbase + u.host_off;
    const size_t mi = std::find(t.models.begin(), t.models.end(), u.model) - t.models.begin();
    const int dev_err = status[mi];
    for (size_t k : u.reqs) {
      Req& q = t.reqs[k];
      if (q.status == XPINN_OK && dev_err)
        fail_req(q, dev_err == XPINN_ERR_TIMEOUT || dev_err == XPINN_ERR_NONFINITE ? dev_err : XPINN_ERR_INVALID,
                 dev_err == XPINN_ERR_NONFINITE ? "a loss became non-finite" : "a device check of the model failed");
    }
    if (u.kind == XPINN_REQ_EVAL) {
      const int row = xp::ctx_out_total(h) * n_comp(u.order);
      const float* hout = reinterpret_cast<const float*>(hp + al256(8 * (size_t)u.n));
      int64_t off = 0;
      for (size_t k : u.reqs) {
        Req& q = t.reqs[k];
        if (q.status == XPINN_OK) memcpy(q.r.out, hout + off * row, sizeof(float) * row * q.r.n);
        off += q.r.n;
        q.batch = (int)u.reqs.size();
      }
    } else if (u.kind == XPINN_REQ_FORK) {
      Req& q = t.reqs[u.reqs[0]];
      const size_t np = (size_t)q.fork_pts;
      const size_t lbytes = 4 * (size_t)q.r.n_steps * q.r.n_sel * XPINN_N_TERMS;
      const char* hl = hp + al256(8 * np) + al256(4 * np);
      if (q.status == XPINN_OK) {
        if (q.r.losses) memcpy(q.r.losses, hl, lbytes);
        if (q.r.params) memcpy(q.r.params, hl + al256(lbytes), 4 * (size_t)q.fork_params);
      }
    } else {
      Req& q = t.reqs[u.reqs[0]];
      if (q.status == XPINN_OK && q.r.losses)
        memcpy(q.r.losses, hp, 4 * (size_t)q.r.n_steps * xp::ctx_n_sub(h) * XPINN_N_TERMS);
    }
  }
  for (Req& q : t.reqs) {
    xpinn_result r;
    memset(&r, 0, sizeof r);
    r.status = q.status;
    r.queue_ms = ms_between(q.t_submit, q.t_admit);
    r.latency_ms = ms_between(q.t_submit, now);
    r.batch = q.batch;
    r.tick_requests = (int32_t)t.reqs.size();
    memcpy(r.error, q.error, sizeof r.error);
    out.emplace_back(q.ticket, r);
  }
}

// Takes pending requests (arrival order) into a new tick while they fit.
bool form_tick(xpinn_server* s, Tick& t) {
  std::vector<Req> take;
  size_t dev = 0, host = 0;
  std::vector<int> models;
  while (!s->pending.empty() && (int)take.size() < MAX_TICK_REQUESTS) {
    const Req& q = s->pending.front();
    const bool new_model = std::find(models.begin(), models.end(), q.r.model) == models.end();
    const size_t host_status = al256(sizeof(int) * (models.size() + (new_model ? 1 : 0)));
    size_t off;
    // would the tick, with this request, fit both rings right now?
    Ring dr = s->dring, hr = s->hring;
    if (!dr.take(dev + q.dev_bytes, off) || !hr.take(host + q.host_bytes + host_status, off)) break;
    dev += q.dev_bytes;
    host += q.host_bytes;
    if (new_model) models.push_back(q.r.model);
    take.push_back(q);
    s->pending.pop_front();
  }
  if (take.empty()) return false;
  t.models = models;
  const size_t host_status = al256(sizeof(int) * models.size());
  t.dev_bytes = dev;
  t.host_bytes = host + host_status;
  s->dring.take(t.dev_bytes, t.dev_off);
  s->hring.take(t.host_bytes, t.host_off);
  const auto now = Clock::now();
  for (Req& q : take) q.t_admit = now;
  t.reqs = std::move(take);
  // units: evaluations grouped by (model, copy, order) in order of first
  // appearance; every other request is its own unit, in arrival order
  size_t doff = 0, hoff = 0;
  std::map<std::tuple<int, int, int>, size_t> group;
  for (size_t i = 0; i < t.reqs.size(); ++i) {
    const xpinn_request& r = t.reqs[i].r;
    if (r.kind == XPINN_REQ_EVAL) {
      const auto key = std::make_tuple(r.model, r.copy, r.order);
      auto it = group.find(key);
      if (it == group.end()) {
        Unit u;
        u.kind = XPINN_REQ_EVAL;
        u.model = r.model;
        u.copy = r.copy;
        u.order = r.order;
        group[key] = t.units.size();
        t.units.push_back(u);
        it = group.find(key);
      }
      Unit& u = t.units[it->second];
      u.reqs.push_back(i);
      u.n += r.n;
    } else {
      Unit u;
      u.kind = r.kind;
      u.model = r.model;
      u.reqs.push_back(i);
      t.units.push_back(u);
    }
  }
  // a merged evaluation needs at most the sum of its requests' footprints
  for (Unit& u : t.units) {
    u.dev_off = doff;
    u.host_off = hoff;
    for (size_t k : u.reqs) {
      doff += t.reqs[k].dev_bytes;
      hoff += t.reqs[k].host_bytes;
    }
  }
  t.status_off = hoff;
  return true;
}

void sched_loop(xpinn_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    // complete finished ticks (in order)
    while (!s->inflight.empty() && tick_done(s->inflight.front())) {
      Tick t = std::move(s->inflight.front());
      s->inflight.pop_front();
      lk.unlock();
      std::vector<std::pair<uint64_t, xpinn_result>> res;
      complete_tick(s, t, res);
      lk.lock();
      s->dring.release_oldest();
      s->hring.release_oldest();
      for (auto& r : res) {
        s->live.erase(r.first);
        s->done[r.first] = r.second;
      }
      s->cv.notify_all();
    }
    if (s->stop && s->pending.empty() && s->inflight.empty()) return;
    // admit and queue a new tick when there is room
    if (!s->pending.empty() && (int)s->inflight.size() < MAX_INFLIGHT_TICKS) {
      Tick t;
      if (form_tick(s, t)) {
        lk.unlock();
        enqueue_tick(s, t);
        lk.lock();
        s->inflight.push_back(std::move(t));
        continue;
      }
    }
    if (s->inflight.empty()) {
      s->cv.wait(lk, [&] { return s->stop || !s->pending.empty(); });
    } else {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
    }
  }
}

int fail(int code, const char* msg) {
  xp::set_last_error(msg);
  return code;
}

}  // namespace

extern "C" {

int xpinn_server_create(const xpinn_handle* models, int32_t n_models, size_t hbm_budget,
                        xpinn_server** out) {
  if (!models || n_models < 1 || !out || hbm_budget < 4096) return fail(XPINN_ERR_INVALID, "bad arguments");
  for (int m = 0; m < n_models; ++m)
    if (!models[m]) return fail(XPINN_ERR_INVALID, "NULL model handle");
  const int dev = xp::ctx_device(models[0]);
  for (int m = 1; m < n_models; ++m)
    if (xp::ctx_device(models[m]) != dev) return fail(XPINN_ERR_UNSUPPORTED, "models on different devices");
  auto* s = new (std::nothrow) xpinn_server();
  if (!s) return fail(XPINN_ERR_OOM, "host allocation failed");
  s->models.assign(models, models + n_models);
  s->budget = hbm_budget;
  s->device = dev;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(dev);
  const size_t host_cap = std::min<size_t>(hbm_budget, (size_t)1 << 30);
  bool ok = cudaMalloc(&s->dev, hbm_budget) == cudaSuccess;
  ok = ok && cudaHostAlloc(&s->host, host_cap, cudaHostAllocDefault) == cudaSuccess;
  for (int i = 0; ok && i < N_STREAMS; ++i)
    ok = cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking) == cudaSuccess;
  cudaSetDevice(prev);
  if (!ok) {
    cudaGetLastError();
    if (s->dev) cudaFree(s->dev);
    if (s->host) cudaFreeHost(s->host);
    for (auto& st : s->streams)
      if (st) cudaStreamDestroy(st);
    delete s;
    return fail(XPINN_ERR_OOM, "could not allocate the server's memory pools");
  }
  s->dring.cap = hbm_budget / 256 * 256;
  s->hring.cap = host_cap / 256 * 256;
  try {
    s->sched = std::thread(sched_loop, s);
  } catch (...) {
    cudaFree(s->dev);
    cudaFreeHost(s->host);
    for (auto& st : s->streams) cudaStreamDestroy(st);
    delete s;
    return fail(XPINN_ERR_INVALID, "could not start the server thread");
  }
  *out = s;
  xp::set_last_error("");
  return XPINN_OK;
}

int xpinn_server_submit(xpinn_server* s, const xpinn_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket) return fail(XPINN_ERR_INVALID, "bad arguments");
  if (req->model < 0 || req->model >= (int)s->models.size()) return fail(XPINN_ERR_INVALID, "bad model");
  xpinn_handle h = s->models[req->model];
  if (req->kind == XPINN_REQ_EVAL) {
    if (req->n < 0 || (req->n > 0 && (!req->xy || !req->out)) || req->order < 0 || req->order > 2 ||
        req->copy < 0 || req->copy >= xp::ctx_n_copies(h))
      return fail(XPINN_ERR_INVALID, "bad evaluation request");
  } else if (req->kind == XPINN_REQ_STEP) {
    if (req->n_steps < 0) return fail(XPINN_ERR_INVALID, "bad step request");
  } else if (req->kind == XPINN_REQ_FORK) {
    if (req->n_steps < 0 || req->n_sel < 1 || !req->sel || !req->n_pts) return fail(XPINN_ERR_INVALID, "bad fork request");
  } else {
    return fail(XPINN_ERR_INVALID, "unknown request kind");
  }
  Req q;
  q.r = *req;
  char msg[160] = {0};
  const int rc = footprint(s, q, msg, sizeof msg);
  if (rc != XPINN_OK) return fail(rc, msg);
  if (q.dev_bytes > s->dring.cap || q.host_bytes + 256 > s->hring.cap)
    return fail(XPINN_ERR_OOM, "request larger than the server's memory pools");
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return fail(XPINN_ERR_INVALID, "server is stopping");
  q.ticket = s->next++;
  q.t_submit = Clock::now();
  q.t_admit = q.t_submit;
  s->pending.push_back(q);
  s->live.insert(q.ticket);
  s->cv.notify_all();
  *ticket = q.ticket;
  xp::set_last_error("");
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
    s->cv.wait(lk, [&] { return s->live.empty(); });
    s->stop = true;
    s->cv.notify_all();
  }
  s->sched.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  for (auto& st : s->streams) cudaStreamDestroy(st);
  cudaFree(s->dev);
  cudaFreeHost(s->host);
  cudaSetDevice(prev);
  delete s;
  return XPINN_OK;
}

}  // extern "C"
