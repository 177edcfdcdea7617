// Continuous-batching request server for BC requests on resident graphs.
//
// Requests (graph, source list, scale, host output) queue in arrival order.
// A background thread admits the head of the queue as soon as two resources
// allow it: GPU residency (the threads its in-flight sources occupy, counted
// against the device's resident-thread capacity) and device memory (its
// per-source slabs plus per-request buffers, counted against a budget fixed at
// server start).  Each admitted request runs as one persistent batched launch
// on its own stream, so requests on different graphs and sizes overlap on the
// device; when one finishes, its slots and memory go to the next in line.  A
// request's share of the GPU is capacity / (requests running or waiting), so
// small requests are not stuck behind a large one for its whole duration.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/bcgpu.h"
#include "bc_common.h"

using namespace bcgpu;

namespace {

using clk = std::chrono::steady_clock;

struct Request {
  bc_request_t id = 0;
  bc_graph* g = nullptr;
  std::vector<uint32_t> sources;
  double scale = 1.0;
  double* out_bc = nullptr;
  int state = BC_REQ_QUEUED;
  int error = BC_OK;
  clk::time_point t_submit, t_done;
  ServeLease* lease = nullptr;
  uint64_t threads = 0;  // resident threads while running
  uint64_t bytes = 0;    // device bytes while running
  int stream_idx = -1;
};

// Requests on the device at once (one stream each), and the number of
// waiting requests the resident threads are shared between.
#ifndef BCGPU_SERVE_STREAMS
#define BCGPU_SERVE_STREAMS 8
#endif
#ifndef BCGPU_SERVE_SHARE
#define BCGPU_SERVE_SHARE 4
#endif
constexpr int kStreams = BCGPU_SERVE_STREAMS;
constexpr size_t kMaxPending = 1 << 20;

struct Server {
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<std::shared_ptr<Request>> pending;
  std::vector<std::shared_ptr<Request>> running;
  std::unordered_map<bc_request_t, std::shared_ptr<Request>> all;
  std::thread th;
  bool started = false, stop = false;
  bc_request_t next_id = 1;
  int device = -1;
  cudaStream_t streams[kStreams] = {};
  bool stream_busy[kStreams] = {};
  uint64_t thread_cap = 0, threads_used = 0;
  uint64_t free_at_start = 0, mem_used = 0;
  // stats
  std::vector<double> lat_ms;
  uint64_t completed = 0, failed = 0, edges = 0;
  uint32_t max_concurrent = 0;

  ~Server() {
    {
      std::lock_guard<std::mutex> lk(mu);
      stop = true;
    }
    cv_sched.notify_all();
    if (th.joinable()) th.join();
  }

  int ensure_started(int dev) {
    if (started) {
      if (dev != device) return set_error(BC_ERR_INVALID, "serving runs on one device per process");
      return BC_OK;
    }
    device = dev;
    cudaError_t e = cudaSetDevice(dev);
    int sms = 0, tpsm = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&tpsm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    for (int i = 0; i < kStreams && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&streams[i], cudaStreamNonBlocking);
    size_t fr = 0, tot = 0;
    if (e == cudaSuccess) e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) return set_error(BC_ERR_CUDA, cudaGetErrorString(e));
    free_at_start = fr;
    thread_cap = (uint64_t)sms * tpsm;
    started = true;
    th = std::thread([this] { loop(); });
    return BC_OK;
  }

  // Device memory the serving slabs may hold: the configured fraction of the
  // memory that was free when the server started.
  uint64_t mem_budget() const {
    bc_config c;
    bc_get_config(&c);
    const double frac = c.mem_fraction > 0 ? c.mem_fraction : 0.6;
    return (uint64_t)(frac * (double)free_at_start);
  }

  // Admission: the head request's slot count from its fair share of the
  // GPU's resident threads, then memory.
  bool try_admit(std::shared_ptr<Request>& r) {
    ServePlan p;
    if (serve_plan(r->g, &p) != BC_OK) {
      r->state = BC_REQ_FAILED;
      r->error = BC_ERR_CUDA;
      return true;
    }
    const uint64_t waiting = running.size() + pending.size();
    const uint64_t share = std::max<uint64_t>(thread_cap / std::max<uint64_t>(1, std::min<uint64_t>(waiting, BCGPU_SERVE_SHARE)), p.team);
    const uint64_t free_threads = thread_cap > threads_used ? thread_cap - threads_used : 0;
    uint64_t slots = std::min<uint64_t>({(uint64_t)std::max<size_t>(r->sources.size(), 1), p.max_slots,
                                         std::min(share, free_threads) / p.team});
    const uint64_t budget = mem_budget();
    const uint64_t free_mem = budget > mem_used ? budget - mem_used : 0;
    if (free_mem < p.fixed_bytes) return false;
    slots = std::min<uint64_t>(slots, (free_mem - p.fixed_bytes) / p.slot_bytes);
    if (slots == 0) return false;
    int si = -1;
    for (int i = 0; i < kStreams; ++i)
      if (!stream_busy[i]) {
        si = i;
        break;
      }
    if (si < 0) return false;
    ServeLease* lease = nullptr;
    const int rc = serve_start(r->g, r->sources.data(), (uint32_t)r->sources.size(), r->scale, (uint32_t)slots,
                               streams[si], &lease);
    if (rc != BC_OK) {
      r->state = BC_REQ_FAILED;
      r->error = rc;
      return true;
    }
    r->lease = lease;
    r->stream_idx = si;
    stream_busy[si] = true;
    r->threads = slots * p.team;
    r->bytes = slots * p.slot_bytes + p.fixed_bytes;
    threads_used += r->threads;
    mem_used += r->bytes;
    r->state = BC_REQ_RUNNING;
    return true;
  }

  void finish(std::shared_ptr<Request>& r) {
    const int rc = serve_finish(r->lease, r->out_bc);
    r->lease = nullptr;
    stream_busy[r->stream_idx] = false;
    threads_used -= r->threads;
    mem_used -= r->bytes;
    r->t_done = clk::now();
    r->state = rc == BC_OK ? BC_REQ_DONE : BC_REQ_FAILED;
    r->error = rc;
    graph_serving_ref(r->g, -1);
    if (rc == BC_OK) {
      ++completed;
      lat_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
      edges += (uint64_t)r->sources.size() * (graph_nnz(r->g) / 2);
    } else {
      ++failed;
    }
  }

  void loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
      bool progressed = false;
      for (size_t i = 0; i < running.size();) {
        if (serve_ready(running[i]->lease)) {
          finish(running[i]);
          running.erase(running.begin() + i);
          progressed = true;
        } else {
          ++i;
        }
      }
      while (!pending.empty()) {
        std::shared_ptr<Request> r = pending.front();
        if (r->state == BC_REQ_CANCELLED) {
          pending.pop_front();
          continue;
        }
        if (!try_admit(r)) break;
        pending.pop_front();
        if (r->state == BC_REQ_RUNNING) {
          running.push_back(r);
          max_concurrent = std::max<uint32_t>(max_concurrent, (uint32_t)running.size());
        } else {
          r->t_done = clk::now();
          ++failed;
          graph_serving_ref(r->g, -1);
        }
        progressed = true;
      }
      if (progressed) cv_done.notify_all();
      if (running.empty() && pending.empty()) {
        cv_sched.wait(lk);
      } else {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(50));
        lk.lock();
      }
    }
  }
};

Server& server() {
  static Server s;
  return s;
}

}  // namespace

extern "C" {

int bc_request_submit(bc_graph_t g, const uint32_t* sources, uint32_t k, double scale, double* out_bc,
                      bc_request_t* out_id) {
  if (!g || !out_bc || !out_id || (k && !sources)) return set_error(BC_ERR_INVALID, "bc_request_submit: bad argument");
  const uint32_t n = graph_n(g);
  for (uint32_t i = 0; i < k; ++i)
    if (sources[i] >= n) return set_error(BC_ERR_INVALID, "bc_request_submit: source out of range");
  Server& s = server();
  std::lock_guard<std::mutex> lk(s.mu);
  if (int rc = s.ensure_started(graph_device(g))) return rc;
  ServePlan p;
  if (int rc = serve_plan(g, &p)) return rc;
  if (p.fixed_bytes + p.slot_bytes > s.mem_budget())
    return set_error(BC_ERR_NOMEM, "bc_request_submit: one source of this graph needs more device memory than the "
                                   "serving budget");
  if (s.pending.size() >= kMaxPending) return set_error(BC_ERR_BUSY, "bc_request_submit: queue full");
  auto r = std::make_shared<Request>();
  r->id = s.next_id++;
  r->g = g;
  r->sources.assign(sources, sources + k);
  r->scale = scale;
  r->out_bc = out_bc;
  r->t_submit = clk::now();
  graph_serving_ref(g, +1);
  s.pending.push_back(r);
  s.all[r->id] = r;
  *out_id = r->id;
  s.cv_sched.notify_all();
  return BC_OK;
}

int bc_request_poll(bc_request_t id, int* out_state) {
  if (!out_state) return set_error(BC_ERR_INVALID, "null out_state");
  Server& s = server();
  std::lock_guard<std::mutex> lk(s.mu);
  auto it = s.all.find(id);
  if (it == s.all.end()) return set_error(BC_ERR_INVALID, "unknown request id");
  *out_state = it->second->state;
  return BC_OK;
}

int bc_request_wait(bc_request_t id, int timeout_ms) {
  Server& s = server();
  std::unique_lock<std::mutex> lk(s.mu);
  auto it = s.all.find(id);
  if (it == s.all.end()) return set_error(BC_ERR_INVALID, "unknown request id");
  std::shared_ptr<Request> r = it->second;
  auto done = [&] { return r->state != BC_REQ_QUEUED && r->state != BC_REQ_RUNNING; };
  if (timeout_ms < 0) {
    s.cv_done.wait(lk, done);
  } else if (!s.cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
    return set_error(BC_ERR_TIMEOUT, "bc_request_wait: timed out");
  }
  s.all.erase(id);
  if (r->state == BC_REQ_DONE) return BC_OK;
  if (r->state == BC_REQ_CANCELLED) return set_error(BC_ERR_CANCELLED, "request cancelled");
  return set_error(r->error ? r->error : BC_ERR_CUDA, "request failed");
}

int bc_request_cancel(bc_request_t id) {
  Server& s = server();
  std::lock_guard<std::mutex> lk(s.mu);
  auto it = s.all.find(id);
  if (it == s.all.end()) return set_error(BC_ERR_INVALID, "unknown request id");
  std::shared_ptr<Request> r = it->second;
  if (r->state == BC_REQ_QUEUED) {
    r->state = BC_REQ_CANCELLED;
    r->t_done = clk::now();
    graph_serving_ref(r->g, -1);
    s.cv_done.notify_all();
    return BC_OK;
  }
  if (r->state == BC_REQ_RUNNING) return set_error(BC_ERR_BUSY, "request already running");
  return BC_OK;
}

int bc_serving_stats_get(bc_serving_stats* out) {
  if (!out) return set_error(BC_ERR_INVALID, "null output");
  Server& s = server();
  std::lock_guard<std::mutex> lk(s.mu);
  memset(out, 0, sizeof *out);
  out->completed = s.completed;
  out->failed = s.failed;
  out->edges_traversed = s.edges;
  out->max_concurrent = s.max_concurrent;
  if (!s.lat_ms.empty()) {
    std::vector<double> v = s.lat_ms;
    std::sort(v.begin(), v.end());
    auto q = [&](double f) { return v[std::min<size_t>(v.size() - 1, (size_t)(f * (v.size() - 1) + 0.5))]; };
    out->p50_ms = q(0.50);
    out->p99_ms = q(0.99);
    double sum = 0;
    for (double x : v) sum += x;
    out->mean_ms = sum / v.size();
  }
  return BC_OK;
}

int bc_serving_reset(void) {
  Server& s = server();
  std::lock_guard<std::mutex> lk(s.mu);
  s.lat_ms.clear();
  s.completed = s.failed = s.edges = 0;
  s.max_concurrent = 0;
  return BC_OK;
}

}  // extern "C"
