// Continuous-batching request server for BC requests on resident graphs.
//
// Requests (graph, source list, scale, host output) queue in arrival order.
// A request is admitted (opened) when device memory allows its workspace:
// per-source slabs for up to as many sources in flight as the GPU holds for
// its graph, its source list and a device accumulator, counted against a
// budget fixed at server start.  Its sources then run as a sequence of source
// batches: each batch is one persistent launch of the batched kernel over
// the next few waves of the request's sources, adding into the accumulator.
// A background thread dispatches batches of all admitted requests, whatever
// their graphs, onto up to 8 streams, so batches of different requests
// overlap on the device and a request's batches interleave with other
// requests' batches.  Before each batch it re-divides the GPU's resident
// threads: a request's share is capacity / min(requests with work left, 2),
// so a large request takes the whole GPU while it runs alone and gives way
// at its next batch boundary when others arrive.  Among requests waiting for
// their next batch, the earliest deadline goes first: submit time + its work
// (sources x entries) / the server's measured throughput, so small requests
// pass large ones, but not ones that have already waited about as long as a
// small request takes (BCGPU_SERVE_ORDER 0: least work left first).  The
// last batch scales the sum and stages it for the caller.
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
  bool cancel = false;  // cancellation asked while RUNNING: ends at the next batch boundary
  clk::time_point t_submit, t_done;
  ServeLease* lease = nullptr;
  ServePlan plan{};
  uint32_t next = 0;       // first source of the next batch
  bool in_batch = false;   // a batch is on the device
  uint64_t threads = 0;    // resident threads of the running batch
  uint64_t bytes = 0;      // device bytes held from open to finish
  int stream_idx = -1;
  uint64_t batch_entries = 0;  // CSR entries the running batch walks (sources x entries)
  double deadline = 0;  // seconds since server start: submit + work / throughput
  // work left, for the dispatch order: sources still to run x CSR entries
  uint64_t work_left() const { return (uint64_t)(sources.size() - next) * std::max<uint64_t>(graph_nnz(g), 1); }
  uint64_t work_total() const { return (uint64_t)sources.size() * std::max<uint64_t>(graph_nnz(g), 1); }
};

// Batches on the device at once (one stream each), the number of requests the
// resident threads are shared between, waves of sources per batch, and the
// number of requests admitted (holding workspaces) at once.
#ifndef BCGPU_SERVE_STREAMS
#define BCGPU_SERVE_STREAMS 8
#endif
#ifndef BCGPU_SERVE_SHARE
#define BCGPU_SERVE_SHARE 2
#endif
#ifndef BCGPU_SERVE_WAVES
#define BCGPU_SERVE_WAVES 2
#endif
#ifndef BCGPU_SERVE_ACTIVE
#define BCGPU_SERVE_ACTIVE 32
#endif
// dispatch order among waiting requests: 1 = earliest deadline, 0 = least work left
#ifndef BCGPU_SERVE_ORDER
#define BCGPU_SERVE_ORDER 1
#endif
constexpr int kStreams = BCGPU_SERVE_STREAMS;
constexpr size_t kMaxPending = 1 << 20;

struct Server {
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<std::shared_ptr<Request>> pending;   // submitted, not admitted
  std::vector<std::shared_ptr<Request>> active;   // admitted: hold a workspace
  std::unordered_map<bc_request_t, std::shared_ptr<Request>> all;
  std::thread th;
  bool started = false, stop = false;
  bc_request_t next_id = 1;
  int device = -1;
  cudaStream_t streams[kStreams] = {};
  bool stream_busy[kStreams] = {};
  cudaStream_t open_stream = nullptr;  // source uploads of newly admitted requests
  uint64_t thread_cap = 0, threads_used = 0;
  uint64_t free_at_start = 0, mem_used = 0;
  // stats
  std::vector<double> lat_ms;
  uint64_t completed = 0, failed = 0, edges = 0, batches = 0;
  uint32_t max_concurrent = 0;
  // throughput estimate for the deadlines: CSR entries walked per second by
  // all batches, an average over windows of about 50 ms with work on the GPU
  clk::time_point t0 = clk::now();
  double entries_per_s = 2e10;
  double win_entries = 0, win_busy_s = 0;
  clk::time_point win_mark = clk::now();
  bool was_busy = false;

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
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&open_stream, cudaStreamNonBlocking);
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

  // A request leaves the server: DONE (result copied out), FAILED or CANCELLED.
  void retire(std::shared_ptr<Request>& r, int state, int rc) {
    if (r->lease) {
      const int frc = serve_finish(r->lease, state == BC_REQ_DONE ? r->out_bc : nullptr);
      if (state == BC_REQ_DONE && frc != BC_OK) {
        state = BC_REQ_FAILED;
        rc = frc;
      }
      r->lease = nullptr;
      mem_used -= r->bytes;
    }
    r->t_done = clk::now();
    r->state = state;
    r->error = rc;
    graph_serving_ref(r->g, -1);
    if (state == BC_REQ_DONE) {
      ++completed;
      lat_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
      edges += (uint64_t)r->sources.size() * (graph_nnz(r->g) / 2);
    } else if (state == BC_REQ_FAILED) {
      ++failed;
    }
  }

  // Admission of the head of the queue: its workspace within the memory budget.
  // Returns false when it has to wait for memory.
  bool try_open(std::shared_ptr<Request>& r) {
    if (serve_plan(r->g, &r->plan) != BC_OK) {
      retire(r, BC_REQ_FAILED, BC_ERR_CUDA);
      return true;
    }
    const ServePlan& p = r->plan;
    uint64_t cap = std::min<uint64_t>((uint64_t)std::max<size_t>(r->sources.size(), 1), p.max_slots);
    const uint64_t budget = mem_budget();
    const uint64_t free_mem = budget > mem_used ? budget - mem_used : 0;
    if (free_mem < p.fixed_bytes + p.slot_bytes) return false;
    cap = std::min<uint64_t>(cap, (free_mem - p.fixed_bytes) / p.slot_bytes);
    ServeLease* lease = nullptr;
    const int rc = serve_open(r->g, r->sources.data(), (uint32_t)r->sources.size(), (uint32_t)cap, open_stream,
                              &lease);
    if (rc != BC_OK) {
      retire(r, BC_REQ_FAILED, rc);
      return true;
    }
    r->lease = lease;
    r->bytes = (uint64_t)serve_slot_cap(lease) * p.slot_bytes + p.fixed_bytes;
    mem_used += r->bytes;
    r->state = BC_REQ_RUNNING;
    r->deadline = std::chrono::duration<double>(r->t_submit - t0).count() + (double)r->work_total() / entries_per_s;
    return true;
  }

  // Throughput estimate: entries of the batches completed in a window over
  // the time the window had batches on the GPU.
  void update_rate(bool busy, double dt) {
    if (busy) win_busy_s += dt;
    if (win_busy_s >= 0.05 && win_entries > 0) {
      const double sample = win_entries / win_busy_s;
      entries_per_s = 0.7 * entries_per_s + 0.3 * sample;
      win_entries = 0;
      win_busy_s = 0;
    }
  }

  // A batch finished: free its threads and stream; the request either goes on,
  // or ends (last batch, error, cancellation).  Returns true when it ended.
  bool batch_done(std::shared_ptr<Request>& r) {
    win_entries += (double)r->batch_entries;
    r->in_batch = false;
    threads_used -= r->threads;
    r->threads = 0;
    stream_busy[r->stream_idx] = false;
    r->stream_idx = -1;
    const int rc = serve_batch_status(r->lease);
    if (rc != BC_OK) {
      retire(r, BC_REQ_FAILED, rc);
      return true;
    }
    if (r->cancel) {
      retire(r, BC_REQ_CANCELLED, BC_ERR_CANCELLED);
      return true;
    }
    if (r->next >= r->sources.size()) {
      retire(r, BC_REQ_DONE, BC_OK);
      return true;
    }
    return false;
  }

  // Next batch of request r on a free stream, within its share of the
  // resident threads.  Returns false when it cannot start now.
  bool dispatch(std::shared_ptr<Request>& r, uint64_t sharers) {
    int si = -1;
    for (int i = 0; i < kStreams; ++i)
      if (!stream_busy[i]) {
        si = i;
        break;
      }
    if (si < 0) return false;
    const ServePlan& p = r->plan;
    const uint64_t share = std::max<uint64_t>(thread_cap / std::max<uint64_t>(1, sharers), p.team);
    const uint64_t free_threads = thread_cap > threads_used ? thread_cap - threads_used : 0;
    const uint32_t left = (uint32_t)(r->sources.size() - r->next);
    const uint64_t slots = std::min<uint64_t>({(uint64_t)serve_slot_cap(r->lease), (uint64_t)std::max(left, 1u),
                                               std::min(share, free_threads) / p.team});
    if (slots == 0) return false;
    const uint32_t count = (uint32_t)std::min<uint64_t>(left, slots * BCGPU_SERVE_WAVES);
    const bool last = r->next + count >= r->sources.size();
    const int rc = serve_batch(r->lease, r->next, count, (uint32_t)slots, last, r->scale, streams[si]);
    if (rc != BC_OK) {
      retire(r, BC_REQ_FAILED, rc);
      return true;
    }
    r->next += count;
    r->batch_entries = (uint64_t)count * std::max<uint64_t>(graph_nnz(r->g), 1);
    r->in_batch = true;
    r->threads = slots * p.team;
    threads_used += r->threads;
    r->stream_idx = si;
    stream_busy[si] = true;
    ++batches;
    return true;
  }

  void loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
      bool progressed = false;
      // 1. finished batches
      for (size_t i = 0; i < active.size();) {
        std::shared_ptr<Request>& r = active[i];
        if (r->in_batch && serve_ready(r->lease)) {
          progressed = true;
          if (batch_done(r)) {
            active.erase(active.begin() + i);
            continue;
          }
        }
        ++i;
      }
      // 2. admission in arrival order, while memory allows
      while (!pending.empty() && active.size() < (size_t)BCGPU_SERVE_ACTIVE) {
        std::shared_ptr<Request> r = pending.front();
        if (r->state == BC_REQ_CANCELLED) {
          pending.pop_front();
          continue;
        }
        if (!try_open(r)) break;
        pending.pop_front();
        if (r->state == BC_REQ_RUNNING) active.push_back(r);
        progressed = true;
      }
      // 3. cancellations of admitted requests between batches, and empty requests
      for (size_t i = 0; i < active.size();) {
        std::shared_ptr<Request>& r = active[i];
        if (!r->in_batch && (r->cancel || r->sources.empty())) {
          if (r->cancel) retire(r, BC_REQ_CANCELLED, BC_ERR_CANCELLED);
          else retire(r, BC_REQ_DONE, serve_batch(r->lease, 0, 0, 1, true, r->scale, open_stream));
          active.erase(active.begin() + i);
          progressed = true;
          continue;
        }
        ++i;
      }
      // 4. next batches: least work left first
      std::vector<std::shared_ptr<Request>> ready;
      uint64_t with_work = 0;
      for (auto& r : active) {
        if (r->next < r->sources.size() || r->in_batch) ++with_work;
        if (!r->in_batch && r->next < r->sources.size()) ready.push_back(r);
      }
      std::stable_sort(ready.begin(), ready.end(), [](const std::shared_ptr<Request>& a,
                                                      const std::shared_ptr<Request>& b) {
        if (BCGPU_SERVE_ORDER == 1 && a->deadline != b->deadline) return a->deadline < b->deadline;
        const uint64_t wa = a->work_left(), wb = b->work_left();
        return wa != wb ? wa < wb : a->id < b->id;
      });
      const uint64_t sharers = std::min<uint64_t>(with_work, BCGPU_SERVE_SHARE);
      for (auto& r : ready) {
        if (r->state != BC_REQ_RUNNING) continue;
        if (dispatch(r, sharers)) progressed = true;
      }
      // requests that failed while dispatching leave the active set
      active.erase(std::remove_if(active.begin(), active.end(),
                                  [](const std::shared_ptr<Request>& r) { return r->state != BC_REQ_RUNNING; }),
                   active.end());
      uint32_t on_device = 0;
      for (auto& r : active) on_device += r->in_batch ? 1u : 0u;
      max_concurrent = std::max(max_concurrent, on_device);
      // the interval since the last mark had batches on the GPU if the last
      // iteration left some there
      const clk::time_point now = clk::now();
      update_rate(was_busy, std::chrono::duration<double>(now - win_mark).count());
      win_mark = now;
      was_busy = on_device > 0;
      if (progressed) cv_done.notify_all();
      if (active.empty() && pending.empty()) {
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
  // a running request stops at its next source-batch boundary; out_bc is not written
  if (r->state == BC_REQ_RUNNING) r->cancel = true;
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
