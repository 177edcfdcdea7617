// C-ABI of libbcgpu (declared in include/bcgpu.h): graph residency, per-source
// slab workspaces, the batched and plain execution paths, the test hook, the
// autotuner and the continuous-batching request server.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/bcgpu.h"
#include "bc_common.h"

using namespace bcgpu;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(BC_ERR_NOMEM, "%s: %s", where, cudaGetErrorString(e));
  }
  return fail(BC_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call)                                         \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

std::mutex g_cfg_mu;
bc_config g_cfg = {BC_MODE_BATCHED, 0, 0, 0, 0, 0, 0.0, 0, 0};

bc_config config_snapshot() {
  std::lock_guard<std::mutex> lk(g_cfg_mu);
  return g_cfg;
}

uint64_t align256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

SlabLayout make_layout(uint32_t n, int dist_bits) {
  SlabLayout L{};
  uint64_t off = 0;
  L.off_d = off;
  off += align256((uint64_t)n * (dist_bits / 8));
  L.off_sig = off;
  off += align256((uint64_t)n * 8);
  L.off_S = off;
  off += align256((uint64_t)n * 4);
  L.off_ends = off;
  off += align256(((uint64_t)n + 2) * 4);
  L.off_near = off;
  off += align256((uint64_t)n * 4);
  L.off_far = off;
  off += align256((uint64_t)n * 4);
  L.off_far2 = off;
  off += align256((uint64_t)n * 4);
  L.off_acc = off;
  off += align256((uint64_t)n * 8);
  L.off_pend = off;
  off += align256(((uint64_t)n + 2) * 4);
  // DAG edge list: 2 n pairs covers every graph whose shortest-path DAG has at
  // most two in-edges per vertex on average (sources beyond it fall back to
  // the per-entry backward scan)
  L.pair_cap = (uint32_t)std::min<uint64_t>(2ull * n + 64, 0xffffffffull);
  L.off_pairs = off;
  off += align256((uint64_t)L.pair_cap * 8);
  L.off_pc = off;
  off += align256((uint64_t)n * 4);
  L.off_pair_e = off;
  off += align256((uint64_t)L.pair_cap * 4);
  L.stride = off;
  return L;
}

// Control block of one launch: source counter, status word, counters, debug.
struct Ctl {
  uint32_t counter;
  int err;
  uint32_t debug[2];
  unsigned long long stats[STAT_COUNT];
};

// Device memory for `slots` sources in flight plus per-call buffers.
struct Workspace {
  uint32_t slots = 0;
  SlabLayout lay{};
  char* slabs = nullptr;
  Ctl* ctl = nullptr;
  double* bc = nullptr;      // [n] (sync paths)
  uint32_t* src = nullptr;   // device copy of the source list
  uint32_t src_cap = 0;
  Ctl* host_ctl = nullptr;   // pinned
  uint32_t* host_src = nullptr;  // pinned staging for sources
  double* host_bc = nullptr;     // pinned staging for results
  cudaEvent_t done = nullptr;
  bool busy = false;
  uint64_t bytes = 0;
};

struct TuneCfg {
  uint32_t team = 0;
  uint64_t width = 0;
  uint32_t settle_in = 0;
  uint32_t max_slots = 0;  // 0: the full resident capacity
  uint32_t warp_deg = 0;
  uint32_t team_deg = 0;
  uint32_t algo = 0;
};

std::mutex g_tune_mu;
std::map<std::string, TuneCfg> g_tune_cache;  // fingerprint -> tuned settings

}  // namespace

struct bc_graph {
  int device = 0;
  uint32_t n = 0;
  uint64_t nnz = 0;
  uint32_t max_w = 0;
  uint64_t width_default = 1;  // mean over non-empty rows of the row's smallest weight (Delta_node)
  int dist_bits = 64;
  int sm_count = 0;
  uint64_t* row_ptr = nullptr;
  uint2* adj = nullptr;
  uint32_t* adjp = nullptr;  // packed 32-bit entries when neighbour and weight fit
  uint32_t col_bits = 0;
  uint32_t* dnode = nullptr;
  uint32_t* dnode2 = nullptr;     // undirected graphs: second smallest incident weight
  uint32_t* dnode_arg = nullptr;  // ... and the neighbour of the smallest
  double* ebc = nullptr;  // lazily allocated [nnz]
  bool relabeled = false;
  bool directed = false;
  uint64_t* in_row_ptr = nullptr;  // directed graphs: in-edge CSR (same entry form)
  uint2* in_adj = nullptr;
  uint32_t* in_adjp = nullptr;
  uint32_t* dnode_in = nullptr;
  uint32_t* o2n = nullptr;  // device maps (relabeled graphs only)
  uint32_t* n2o = nullptr;
  uint32_t* e2o = nullptr;
  uint32_t* esm = nullptr;  // edge output: walked entry -> caller's output entry (built on first use)
  int esm_state = 0;        // 0 not built, 1 ready, 2 unavailable (an entry without a twin)
  std::vector<uint32_t> h_o2n;  // host copy of old -> new
  uint64_t device_bytes = 0;
  std::string fingerprint;
  TuneCfg tuned;
  std::mutex mu;  // guards the workspace pool and stats
  std::vector<std::unique_ptr<Workspace>> pool;
  std::unordered_map<cudaStream_t, Workspace*> async_ws;
  bc_run_stats last{};
  std::atomic<int> serving_refs{0};
  std::atomic<int> step_refs{0};
  PlainWork* plain = nullptr;
  PaperWork* paper = nullptr;
  cudaStream_t stream = nullptr;  // internal stream of the synchronous calls
};

namespace {

GraphDev view(const bc_graph* g) {
  GraphDev v;
  v.n = g->n;
  v.nnz = g->nnz;
  v.row_ptr = g->row_ptr;
  v.adj = g->adj;
  v.adjp = g->adjp;
  v.col_bits = g->col_bits;
  v.dnode = g->dnode;
  v.dnode2 = g->dnode2;
  v.dnode_arg = g->dnode_arg;
  v.o2n = g->o2n;
  v.n2o = g->n2o;
  v.e2o = g->e2o;
  v.in_row_ptr = g->in_row_ptr;
  v.in_adj = g->in_adj;
  v.in_adjp = g->in_adjp;
  v.dnode_in = g->dnode_in;
  return v;
}

void ws_free(Workspace* w) {
  if (!w) return;
  cudaFree(w->slabs);
  cudaFree(w->ctl);
  cudaFree(w->bc);
  cudaFree(w->src);
  if (w->host_ctl) cudaFreeHost(w->host_ctl);
  if (w->host_src) cudaFreeHost(w->host_src);
  if (w->host_bc) cudaFreeHost(w->host_bc);
  if (w->done) cudaEventDestroy(w->done);
}

// Settings for a run: explicit config fields win, then the graph's tuned
// values, then heuristics.
// Default L2 evict-last prefix (vertex ids after degree relabeling).
#ifndef BCGPU_HOT_VERTICES
#define BCGPU_HOT_VERTICES 32768u
#endif

struct RunCfg {
  uint32_t team;
  uint64_t width;
  uint32_t settle_in;
  uint32_t refine;  // settled-neighbour refinement of Delta_node (undirected graphs)
  uint64_t phase_cap;
  uint32_t max_slots;
  double mem_fraction;
  uint32_t mode;
  uint32_t warp_deg;
  uint32_t team_deg;
  uint32_t algo;  // ALGO_STRICT or ALGO_DELTA
  uint32_t hot_n;
};

RunCfg resolve(const bc_graph* g) {
  bc_config c = config_snapshot();
  RunCfg r;
  r.mode = c.mode;
  // entries walked per vertex: a directed graph's batches walk in- and out-edges
  const double avg_deg = g->n ? (double)g->nnz * (g->directed ? 2.0 : 1.0) / g->n : 0.0;
  // measured defaults: the widest CTA teams for dense skewed graphs (large
  // frontiers per batch; half as many sources in flight keeps more of each
  // source's distance array in L2), 128-thread teams for sparse high-diameter
  // graphs
  const uint32_t wide = g->dist_bits == 32 ? 1024u : 512u;
  const uint32_t team_default = avg_deg >= 20.0 ? wide : (avg_deg >= 6.0 ? 256u : 128u);
  r.team = c.team_threads ? c.team_threads : (g->tuned.team ? g->tuned.team : team_default);
  if (r.team == 1024 && g->dist_bits != 32) r.team = 512;  // 1024-thread teams hold 32-bit distances only
  r.width = c.bucket_width ? c.bucket_width
                           : (g->tuned.width ? g->tuned.width : g->width_default);
  // 1: OUT or IN with the settled-neighbour refinement; 2: OUT alone with
  // Delta_node (the paper's test); 3: OUT or IN with Delta_node (the default
  // until the autotuner has timed the refinement for this graph)
  uint32_t si = c.settle_in ? c.settle_in : (g->tuned.settle_in ? g->tuned.settle_in : 3u);
  r.settle_in = (si == 1u || si == 3u) ? 1u : 0u;
  r.refine = (si == 1u && g->dnode2 != nullptr) ? 1u : 0u;
  // phases <= n (each settles at least the smallest candidate), refills that
  // move entries <= n per queue level, empty refills <= second-level refills + 2:
  // phases + refills <= 4n + 2 (delta-stepping rounds + advances <= 3n)
  r.phase_cap = c.phase_cap ? c.phase_cap : 4ull * g->n + 64;
  r.max_slots = c.max_slots ? c.max_slots : g->tuned.max_slots;
  r.mem_fraction = c.mem_fraction > 0 ? c.mem_fraction : 0.6;
  r.warp_deg = c.warp_degree ? c.warp_degree : (g->tuned.warp_deg ? g->tuned.warp_deg : 32u);
  r.team_deg = c.team_degree ? c.team_degree : (g->tuned.team_deg ? g->tuned.team_deg : 8u * r.team);
  r.team_deg = std::max(r.team_deg, r.warp_deg);
  const uint32_t al = c.algorithm ? c.algorithm : (g->tuned.algo ? g->tuned.algo : (uint32_t)BC_ALGO_STRICT);
  r.algo = (al == BC_ALGO_DELTA) ? ALGO_DELTA : ALGO_STRICT;
  const uint32_t hot = c.hot_vertices ? c.hot_vertices : BCGPU_HOT_VERTICES;
  r.hot_n = g->relabeled ? std::min<uint32_t>(g->n, hot) : 0u;
  return r;
}

// Number of sources in flight for a run of k sources.
int plan_slots(const bc_graph* g, const RunCfg& r, uint32_t k, uint32_t* slots_out) {
  int bps = 0;
  cudaError_t e = batched_occupancy(g->dist_bits, (int)r.team, (int)r.algo, &bps);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  const uint32_t per_block = (uint32_t)(batched_block_threads((int)r.team) / (int)r.team);
  uint64_t slots = (uint64_t)std::max(bps, 1) * g->sm_count * per_block;
  size_t free_b = 0, total_b = 0;
  CK(cudaMemGetInfo(&free_b, &total_b));
  const uint64_t stride = make_layout(g->n, g->dist_bits).stride;
  const uint64_t by_mem = (uint64_t)((double)free_b * r.mem_fraction) / std::max<uint64_t>(stride, 1);
  slots = std::min<uint64_t>(slots, by_mem);
  if (r.max_slots) slots = std::min<uint64_t>(slots, r.max_slots);
  slots = std::min<uint64_t>(slots, std::max<uint32_t>(k, 1));
  if (slots == 0) return fail(BC_ERR_NOMEM, "device memory too small for one per-source slab (%llu bytes)",
                              (unsigned long long)stride);
  *slots_out = (uint32_t)slots;
  return BC_OK;
}

// Acquire a free workspace with >= slots slabs and a source buffer >= k.
// The caller's stream waits for the workspace's previous use.
int ws_acquire(bc_graph* g, uint32_t slots, uint32_t k, cudaStream_t st, Workspace** out) {
  Workspace* w = nullptr;
  {
    std::lock_guard<std::mutex> lk(g->mu);
    for (auto& p : g->pool)
      if (!p->busy && p->slots >= slots && (!w || p->slots < w->slots)) w = p.get();
    if (w) w->busy = true;
  }
  if (!w) {
    auto nw = std::make_unique<Workspace>();
    nw->slots = slots;
    nw->lay = make_layout(g->n, g->dist_bits);
    const uint64_t bytes = nw->lay.stride * slots;
    cudaError_t e = cudaMalloc(&nw->slabs, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&nw->ctl, sizeof(Ctl));
    if (e == cudaSuccess) e = cudaMalloc(&nw->bc, (size_t)g->n * 8);
    if (e == cudaSuccess) e = cudaMallocHost(&nw->host_ctl, sizeof(Ctl));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&nw->done, cudaEventDisableTiming);
    // the slab invariant: every distance word is INF between sources
    // and the backward accumulators are zero; other arrays are written before read
    if (e == cudaSuccess)
      e = launch_fill_slabs(nw->slabs, nw->lay.stride, slots, nw->lay.off_d,
                            align256((uint64_t)g->n * (g->dist_bits / 8)), 0xffffffffu, st);
    if (e == cudaSuccess)
      e = launch_fill_slabs(nw->slabs, nw->lay.stride, slots, nw->lay.off_acc, align256((uint64_t)g->n * 8), 0u, st);
    if (e == cudaSuccess)
      e = launch_fill_slabs(nw->slabs, nw->lay.stride, slots, nw->lay.off_pc, align256((uint64_t)g->n * 4), 0u, st);
    if (e != cudaSuccess) {
      ws_free(nw.get());
      return cuda_fail(e, "workspace allocation");
    }
    nw->bytes = bytes;
    nw->busy = true;
    w = nw.get();
    std::lock_guard<std::mutex> lk(g->mu);
    g->pool.push_back(std::move(nw));
  } else {
    CK(cudaStreamWaitEvent(st, w->done, 0));
  }
  if (w->src_cap < k) {
    // previous uses of this workspace are ordered before st; free is safe after a sync
    cudaError_t e = cudaSuccess;
    if (w->src) {
      e = cudaStreamSynchronize(st);
      if (e == cudaSuccess) {
        cudaFree(w->src);
        cudaFreeHost(w->host_src);
        w->src = nullptr;
        w->host_src = nullptr;
        w->src_cap = 0;
      }
    }
    const uint32_t cap = std::max<uint32_t>(k, 1024);
    if (e == cudaSuccess) e = cudaMalloc(&w->src, (size_t)cap * 4);
    if (e == cudaSuccess) e = cudaMallocHost(&w->host_src, (size_t)cap * 4);
    if (e != cudaSuccess) {
      // hand the workspace back (without a source buffer) so the pool stays usable
      if (w->src && !w->host_src) {
        cudaFree(w->src);
        w->src = nullptr;
      }
      std::lock_guard<std::mutex> lk(g->mu);
      w->busy = false;
      return cuda_fail(e, "workspace source buffer");
    }
    w->src_cap = cap;
  }
  *out = w;
  return BC_OK;
}

void ws_release(bc_graph* g, Workspace* w, cudaStream_t st) {
  cudaEventRecord(w->done, st);
  std::lock_guard<std::mutex> lk(g->mu);
  w->busy = false;
}

// Edge output over the DAG edge list needs, for every entry the forward pass
// walks (out-entries of an undirected graph, in-entries of a directed one),
// the caller's index of the entry that carries its share: the twin u -> v of
// the walked entry v -> u, or the out-entry u -> v of the in-entry.  Built on
// the host from the device CSR on the first edge-output call; a graph whose
// undirected entries lack twins keeps the per-entry backward scan.
int ensure_edge_map(bc_graph* g) {
  {
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->esm_state) return BC_OK;
  }
  const uint32_t n = g->n;
  const uint64_t nnz = g->nnz;
  std::vector<uint64_t> rp((size_t)n + 1);
  std::vector<uint32_t> col(nnz), wt(nnz), e2o;
  CK(cudaMemcpy(rp.data(), g->row_ptr, ((size_t)n + 1) * 8, cudaMemcpyDeviceToHost));
  if (g->adjp) {
    std::vector<uint32_t> p(nnz);
    if (nnz) CK(cudaMemcpy(p.data(), g->adjp, nnz * 4, cudaMemcpyDeviceToHost));
    const uint32_t mask = (g->col_bits >= 32) ? 0xffffffffu : ((1u << g->col_bits) - 1u);
    for (uint64_t e = 0; e < nnz; ++e) {
      col[e] = p[e] & mask;
      wt[e] = p[e] >> g->col_bits;
    }
  } else {
    std::vector<uint2> p(nnz);
    if (nnz) CK(cudaMemcpy(p.data(), g->adj, nnz * 8, cudaMemcpyDeviceToHost));
    for (uint64_t e = 0; e < nnz; ++e) {
      col[e] = p[e].x;
      wt[e] = p[e].y;
    }
  }
  if (g->e2o) {
    e2o.resize(nnz);
    if (nnz) CK(cudaMemcpy(e2o.data(), g->e2o, nnz * 4, cudaMemcpyDeviceToHost));
  }
  auto out_id = [&](uint64_t e) { return g->e2o ? e2o[e] : (uint32_t)e; };
  std::vector<uint32_t> map(std::max<uint64_t>(nnz, 1), 0);
  bool ok = true;
  if (g->directed) {
    // in-entry order of the transpose built at creation: rows by target,
    // within a row by source (the out-CSR's row order)
    std::vector<uint64_t> fill((size_t)n + 1, 0);
    for (uint64_t e = 0; e < nnz; ++e) ++fill[(size_t)col[e] + 1];
    for (uint32_t v = 0; v < n; ++v) fill[v + 1] += fill[v];
    for (uint32_t v = 0; v < n; ++v)
      for (uint64_t e = rp[v]; e < rp[v + 1]; ++e) map[fill[col[e]]++] = out_id(e);
  } else {
    // each row sorted by (neighbour, weight, entry); the k-th entry v -> u of
    // weight w pairs with the k-th entry u -> v of weight w
    std::vector<uint32_t> perm(nnz);
    for (uint64_t e = 0; e < nnz; ++e) perm[e] = (uint32_t)e;
    auto less = [&](uint32_t x, uint32_t y) {
      return col[x] != col[y] ? col[x] < col[y] : (wt[x] != wt[y] ? wt[x] < wt[y] : x < y);
    };
    for (uint32_t v = 0; v < n; ++v) std::sort(perm.begin() + rp[v], perm.begin() + rp[v + 1], less);
    for (uint32_t a = 0; a < n && ok; ++a) {
      uint64_t group = rp[a];
      for (uint64_t i = rp[a]; i < rp[a + 1]; ++i) {
        const uint32_t e = perm[i];
        if (i > rp[a] && (col[perm[i - 1]] != col[e] || wt[perm[i - 1]] != wt[e])) group = i;
        const uint64_t k = i - group;
        const uint32_t b = col[e], w = wt[e];
        auto first = std::lower_bound(perm.begin() + rp[b], perm.begin() + rp[b + 1], 0u,
                                      [&](uint32_t x, uint32_t) { return col[x] != a ? col[x] < a : wt[x] < w; });
        const uint64_t pos = (uint64_t)(first - perm.begin()) + k;
        if (pos >= rp[b + 1] || col[perm[pos]] != a || wt[perm[pos]] != w) {
          ok = false;
          break;
        }
        map[e] = out_id(perm[pos]);
      }
    }
  }
  uint32_t* d_map = nullptr;
  if (ok) {
    CK(cudaMalloc(&d_map, std::max<uint64_t>(nnz, 1) * 4));
    cudaError_t e = nnz ? cudaMemcpy(d_map, map.data(), nnz * 4, cudaMemcpyHostToDevice) : cudaSuccess;
    if (e != cudaSuccess) {
      cudaFree(d_map);
      return cuda_fail(e, "edge map upload");
    }
  }
  std::lock_guard<std::mutex> lk(g->mu);
  if (g->esm_state) {  // built concurrently by another thread
    cudaFree(d_map);
    return BC_OK;
  }
  g->esm = d_map;
  g->esm_state = ok ? 1 : 2;
  return BC_OK;
}

BatchArgs make_args(bc_graph* g, Workspace* w, const RunCfg& r, const uint32_t* d_src, uint32_t k, double* d_bc,
                    double* d_ebc, uint32_t slots, uint32_t flags) {
  BatchArgs a{};
  a.g = view(g);
  a.sources = d_src;
  a.k = k;
  a.counter = &w->ctl->counter;
  a.bc = d_bc;
  a.ebc = d_ebc;
  a.slabs = w->slabs;
  a.lay = w->lay;
  a.nslots = slots;
  a.width = r.width;
  a.settle_in = r.settle_in;
  a.refine = r.refine;
  a.phase_cap = r.phase_cap;
  a.err = &w->ctl->err;
  a.stats = w->ctl->stats;
  a.flags = flags;
  a.debug_out = w->ctl->debug;
  a.warp_deg = r.warp_deg;
  a.team_deg = r.team_deg;
  a.algo = r.algo;
  a.esm = (d_ebc && g->esm_state == 1) ? g->esm : nullptr;
  // the highest-degree vertices after relabeling: 128 KiB of 32-bit distance
  // words per source (the whole L2 holds this prefix for ~1000 sources)
  a.hot_n = r.hot_n;
  return a;
}

int grid_for_slots(uint32_t team, uint32_t slots) {
  const uint32_t per_block = (uint32_t)(batched_block_threads((int)team) / (int)team);
  return (int)((slots + per_block - 1) / per_block);
}

// Enqueue one batched run: zero the output and control block, launch, scale.
int enqueue_batched(bc_graph* g, Workspace* w, const RunCfg& r, const uint32_t* d_src, uint32_t k, double scale,
                    double* d_bc, double* d_ebc, uint32_t slots, uint32_t flags, cudaStream_t st, bool check_src) {
  CK(cudaMemsetAsync(w->ctl, 0, sizeof(Ctl), st));
  if (d_bc) CK(cudaMemsetAsync(d_bc, 0, (size_t)g->n * 8, st));
  if (d_ebc) CK(cudaMemsetAsync(d_ebc, 0, (size_t)g->nnz * 8, st));
  if (check_src) CK(launch_check_sources(d_src, k, g->n, &w->ctl->err, st));
  BatchArgs a = make_args(g, w, r, d_src, k, d_bc, d_ebc, slots, flags);
  CK(launch_batched(a, g->dist_bits, (int)r.team, grid_for_slots(r.team, slots), st));
  if (d_bc && scale != 1.0) CK(launch_scale(d_bc, g->n, scale, st));
  if (d_ebc && scale != 1.0) CK(launch_scale(d_ebc, g->nnz, scale, st));
  return BC_OK;
}

int status_from_dev(int dev) {
  if (dev == DEV_OK) return BC_OK;
  if (dev == DEV_ERR_TIMEOUT) return fail(BC_ERR_TIMEOUT, "device phase cap reached (BC_ERR_TIMEOUT)");
  if (dev == DEV_ERR_INVALID) return fail(BC_ERR_INVALID, "a source is out of range");
  if (dev == DEV_ERR_INTERNAL) return fail(BC_ERR_CUDA, "device consistency check failed (DAG levels do not cover the reached set)");
  return fail(BC_ERR_CUDA, "unknown device status %d", dev);
}

void record_stats(bc_graph* g, const Ctl& c, const RunCfg& r, uint32_t slots) {
  std::lock_guard<std::mutex> lk(g->mu);
  g->last.sources = c.stats[STAT_SOURCES];
  g->last.phases = c.stats[STAT_PHASES];
  g->last.refills = c.stats[STAT_REFILLS];
  g->last.reached = c.stats[STAT_REACHED];
  g->last.relax_atomics = c.stats[STAT_RELAX];
  g->last.entries_scanned = c.stats[STAT_ENTRIES];
  g->last.dag_edges = c.stats[STAT_DAG_EDGES];
  g->last.pair_overflows = c.stats[STAT_PAIR_OVERFLOW];
  g->last.cycles_expand = c.stats[STAT_CYC_EXPAND];
  g->last.cycles_refill = c.stats[STAT_CYC_REFILL];
  g->last.cycles_settle = c.stats[STAT_CYC_SETTLE];
  g->last.cycles_backward = c.stats[STAT_CYC_BACKWARD];
  g->last.near_scanned = c.stats[STAT_NEAR_SCANNED];
  g->last.far_scanned = c.stats[STAT_FAR_SCANNED];
  g->last.levels = c.stats[STAT_LEVELS];
  g->last.algorithm = r.algo == ALGO_DELTA ? BC_ALGO_DELTA : BC_ALGO_STRICT;
  g->last.team_threads = r.team;
  g->last.slots = slots;
  g->last.bucket_width = r.width;
  g->last.warp_degree = r.warp_deg;
  g->last.team_degree = r.team_deg;
  g->last.settle_in = r.settle_in ? (r.refine ? 1u : 3u) : 2u;
}

int check_graph(bc_graph_t g) {
  if (!g) return fail(BC_ERR_INVALID, "null graph handle");
  return BC_OK;
}

// Synchronous batched run with host sources and host outputs.
int compute_sync(bc_graph* g, const uint32_t* sources, uint32_t k, double scale, double* out_bc, double* out_ebc,
                 const RunCfg& r) {
  for (uint32_t i = 0; i < k; ++i)
    if (sources[i] >= g->n) return fail(BC_ERR_INVALID, "source %u out of range (n = %u)", sources[i], g->n);
  if (out_ebc)
    if (int rc = ensure_edge_map(g)) return rc;
  cudaStream_t st = g->stream;
  uint32_t slots = 0;
  int rc = plan_slots(g, r, k, &slots);
  if (rc) return rc;
  Workspace* w = nullptr;
  if ((rc = ws_acquire(g, slots, k, st, &w))) return rc;
  if (k) {
    memcpy(w->host_src, sources, (size_t)k * 4);
    cudaError_t e = cudaMemcpyAsync(w->src, w->host_src, (size_t)k * 4, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      ws_release(g, w, st);
      return cuda_fail(e, "cudaMemcpyAsync(sources)");
    }
  }
  double* d_ebc = nullptr;
  if (out_ebc) {
    if (!g->ebc) {
      cudaError_t e = cudaMalloc(&g->ebc, (size_t)std::max<uint64_t>(g->nnz, 1) * 8);
      if (e != cudaSuccess) {
        ws_release(g, w, st);
        return cuda_fail(e, "cudaMalloc(edge bc)");
      }
    }
    d_ebc = g->ebc;
  }
  rc = enqueue_batched(g, w, r, w->src, k, scale, w->bc, d_ebc, slots, 0, st, false);
  if (rc) {
    ws_release(g, w, st);
    return rc;
  }
  cudaError_t e = cudaMemcpyAsync(w->host_ctl, w->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && out_bc) e = cudaMemcpyAsync(out_bc, w->bc, (size_t)g->n * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && out_ebc && g->nnz)
    e = cudaMemcpyAsync(out_ebc, d_ebc, (size_t)g->nnz * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  const Ctl c = *w->host_ctl;  // read before the workspace goes back to the pool
  ws_release(g, w, st);
  if (e != cudaSuccess) return cuda_fail(e, "batched run");
  record_stats(g, c, r, slots);
  return status_from_dev(c.err);
}

int compute_plain(bc_graph* g, const uint32_t* sources, uint32_t k, double scale, double* out_bc, const RunCfg& r) {
  if (g->directed) return fail(BC_ERR_INVALID, "BC_MODE_PLAIN runs undirected graphs only");
  for (uint32_t i = 0; i < k; ++i)
    if (sources[i] >= g->n) return fail(BC_ERR_INVALID, "source %u out of range (n = %u)", sources[i], g->n);
  cudaStream_t st = g->stream;
  if (!g->plain) {
    cudaError_t e;
    g->plain = plain_create(g->n, g->dist_bits, &e);
    if (!g->plain) return cuda_fail(e, "plain workspace");
  }
  double* d_bc = nullptr;
  CK(cudaMalloc(&d_bc, (size_t)g->n * 8));
  cudaError_t e = cudaMemsetAsync(d_bc, 0, (size_t)g->n * 8, st);
  int dev = DEV_OK;
  unsigned long long stats[STAT_COUNT] = {0};
  if (e == cudaSuccess)
    e = plain_run(g->plain, view(g), g->dist_bits, sources, g->relabeled ? g->h_o2n.data() : nullptr, k, d_bc,
                  r.width, r.settle_in, r.phase_cap, g->sm_count, st, &dev, stats);
  if (e == cudaSuccess && scale != 1.0) e = launch_scale(d_bc, g->n, scale, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_bc, d_bc, (size_t)g->n * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d_bc);
  if (e != cudaSuccess) return cuda_fail(e, "plain run");
  Ctl c{};
  memcpy(c.stats, stats, sizeof stats);
  record_stats(g, c, r, 1);
  return status_from_dev(dev);
}

// 64-bit finaliser of SplitMix64 (Steele, Lea and Flood, OOPSLA 2014).
uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// True when the multiset of entries (v -> u, w) equals that of their reverses
// (u -> v, w), compared through a sum mod 2^64 of a hash of each entry: exact
// for a symmetric CSR, and an asymmetric one passes only with probability about
// 2^-64.  O(nnz).
bool symmetric_by_hash(uint32_t n, const uint64_t* rp, const uint32_t* col, const uint32_t* w) {
  uint64_t fwd = 0, rev = 0;
  for (uint32_t v = 0; v < n; ++v)
    for (uint64_t e = rp[v]; e < rp[v + 1]; ++e) {
      const uint64_t hw = mix64((uint64_t)w[e] + 0x9e3779b97f4a7c15ull);
      fwd += mix64((((uint64_t)v << 32) | col[e]) ^ hw);
      rev += mix64((((uint64_t)col[e] << 32) | v) ^ hw);
    }
  return fwd == rev;
}

// Upper bound on every finite shortest-path distance of a symmetric graph:
// within a component, two vertices are joined through the vertex r its
// breadth-first search starts from by a path of at most 2 ecc(r) edges (ecc =
// hop eccentricity), each of weight at most max_w.  O(n + nnz).
uint64_t hop_distance_bound(uint32_t n, const uint64_t* rp, const uint32_t* col, uint32_t max_w) {
  std::vector<uint32_t> hop(n, 0xffffffffu), q(n);
  uint64_t max_ecc = 0;
  for (uint32_t r = 0; r < n; ++r) {
    if (hop[r] != 0xffffffffu) continue;
    uint32_t head = 0, tail = 0;
    hop[r] = 0;
    q[tail++] = r;
    while (head < tail) {
      const uint32_t v = q[head++];
      for (uint64_t e = rp[v]; e < rp[v + 1]; ++e) {
        const uint32_t u = col[e];
        if (hop[u] == 0xffffffffu) {
          hop[u] = hop[v] + 1;
          q[tail++] = u;
        }
      }
    }
    max_ecc = std::max<uint64_t>(max_ecc, hop[q[tail - 1]]);
  }
  return 2ull * max_ecc * std::max<uint32_t>(max_w, 1);
}

// Distance word width.  32 bits when every value the kernels form fits with
// room to spare: a finite distance D, a tentative distance D + w and a
// threshold key D + 2 max_w stay below half of the 32-bit INF word.  D is
// bounded by (n - 1) max_w for any graph, and for symmetric undirected graphs
// also by the hop bound above (the 1024 x 1024 grid with weights up to 10^4:
// about 5 * 10^7 against 10^10).
int distance_bits(uint32_t n, const uint64_t* rp, const uint32_t* col, const uint32_t* w, uint32_t max_w,
                  bool directed) {
  const uint64_t mw = std::max<uint32_t>(max_w, 1);
  const uint64_t half = 0x7fffffffull;
  if ((uint64_t)n * mw + 2 * mw < half) return 32;
  if (directed || !symmetric_by_hash(n, rp, col, w)) return 64;
  const uint64_t bound = hop_distance_bound(n, rp, col, max_w);
  return bound + 2 * mw < half ? 32 : 64;
}

std::string fingerprint(uint32_t n, uint64_t nnz, const uint64_t* rp, const uint32_t* col, const uint32_t* w) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](uint64_t x) {
    h ^= x;
    h *= 1099511628211ull;
  };
  mix(n);
  mix(nnz);
  const uint64_t step = std::max<uint64_t>(1, nnz / 4096);
  for (uint64_t e = 0; e < nnz; e += step) {
    mix(col[e]);
    mix(w[e]);
  }
  const uint64_t vstep = std::max<uint64_t>(1, n / 4096);
  for (uint64_t v = 0; v <= n; v += vstep) mix(rp[v]);
  char buf[64];
  snprintf(buf, sizeof buf, "%u-%llu-%016llx", n, (unsigned long long)nnz, (unsigned long long)h);
  return buf;
}

}  // namespace

int bcgpu::set_error(int code, const char* msg) { return fail(code, "%s", msg); }

// ------------------------------------------------------------- serving glue

struct bcgpu::ServeLease {
  bc_graph* g;
  Workspace* w;
  cudaStream_t st;   // stream of the latest source batch
  cudaEvent_t ev;    // recorded after each source batch
  uint32_t k;
  uint32_t slot_cap;  // slabs the lease holds
};

int bcgpu::graph_device(const bc_graph* g) { return g->device; }
uint32_t bcgpu::graph_n(const bc_graph* g) { return g->n; }
uint64_t bcgpu::graph_nnz(const bc_graph* g) { return g->nnz; }
void bcgpu::graph_serving_ref(bc_graph* g, int delta) { g->serving_refs += delta; }

int bcgpu::serve_plan(bc_graph* g, ServePlan* out) {
  RunCfg r = resolve(g);
  int bps = 0;
  cudaError_t e = batched_occupancy(g->dist_bits, (int)r.team, (int)r.algo, &bps);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy");
  const uint32_t per_block = (uint32_t)(batched_block_threads((int)r.team) / (int)r.team);
  out->team = r.team;
  out->max_slots = (uint32_t)std::max(bps, 1) * (uint32_t)g->sm_count * per_block;
  out->slot_bytes = make_layout(g->n, g->dist_bits).stride;
  out->fixed_bytes = (uint64_t)g->n * 16 + 4096;
  return BC_OK;
}

int bcgpu::serve_open(bc_graph* g, const uint32_t* sources, uint32_t k, uint32_t slot_cap, cudaStream_t st,
                      ServeLease** out) {
  Workspace* w = nullptr;
  const uint32_t cap = std::max<uint32_t>(slot_cap, 1);
  int rc = ws_acquire(g, cap, k, st, &w);
  if (rc) return rc;
  cudaError_t e = cudaSuccess;
  if (!w->host_bc) e = cudaMallocHost(&w->host_bc, (size_t)g->n * 8);
  // the request's sources and its zeroed accumulator, ordered before its first source batch on st
  if (e == cudaSuccess && k) {
    memcpy(w->host_src, sources, (size_t)k * 4);
    e = cudaMemcpyAsync(w->src, w->host_src, (size_t)k * 4, cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(w->bc, 0, (size_t)g->n * 8, st);
  // the first batch, on whichever stream, waits for this event
  if (e == cudaSuccess) e = cudaEventRecord(w->done, st);
  if (e != cudaSuccess) {
    ws_release(g, w, st);
    return cuda_fail(e, "serve_open");
  }
  *out = new ServeLease{g, w, st, w->done, k, std::min(cap, w->slots)};
  return BC_OK;
}

uint32_t bcgpu::serve_slot_cap(const ServeLease* l) { return l->slot_cap; }

int bcgpu::serve_batch(ServeLease* l, uint32_t first, uint32_t count, uint32_t slots, bool last, double scale,
                       cudaStream_t st) {
  bc_graph* g = l->g;
  Workspace* w = l->w;
  RunCfg r = resolve(g);
  r.mode = BC_MODE_BATCHED;
  l->st = st;
  // the previous batch of this request (possibly on another stream) comes first
  cudaError_t e = cudaStreamWaitEvent(st, w->done, 0);
  if (e == cudaSuccess) e = cudaMemsetAsync(w->ctl, 0, sizeof(Ctl), st);
  const uint32_t sl = std::max<uint32_t>(1, std::min<uint32_t>(slots, l->slot_cap));
  if (e == cudaSuccess) {
    BatchArgs a = make_args(g, w, r, w->src + first, count, w->bc, nullptr, sl, 0);
    e = launch_batched(a, g->dist_bits, (int)r.team, grid_for_slots(r.team, sl), st);
  }
  if (e == cudaSuccess && last && scale != 1.0) e = launch_scale(w->bc, g->n, scale, st);
  if (e == cudaSuccess && last)
    e = cudaMemcpyAsync(w->host_bc, w->bc, (size_t)g->n * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w->host_ctl, w->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
  // recorded even after a failed enqueue, so the workspace is released only
  // once whatever did get enqueued has run
  const cudaError_t er = cudaEventRecord(w->done, st);
  if (e == cudaSuccess) e = er;
  if (e != cudaSuccess) return cuda_fail(e, "serving batch");
  return BC_OK;
}

int bcgpu::serve_batch_status(ServeLease* l) {
  cudaError_t e = cudaEventSynchronize(l->ev);
  if (e != cudaSuccess) return cuda_fail(e, "serving batch");
  return status_from_dev(l->w->host_ctl->err);
}

bool bcgpu::serve_ready(ServeLease* l) { return cudaEventQuery(l->ev) != cudaErrorNotReady; }

int bcgpu::serve_finish(ServeLease* l, double* out_bc) {
  cudaError_t e = cudaEventSynchronize(l->ev);
  int rc = BC_OK;
  if (e != cudaSuccess) {
    rc = cuda_fail(e, "serving run");
  } else if (out_bc) {
    memcpy(out_bc, l->w->host_bc, (size_t)l->g->n * 8);
    rc = status_from_dev(l->w->host_ctl->err);
  }
  {
    std::lock_guard<std::mutex> lk(l->g->mu);
    l->w->busy = false;
  }
  delete l;
  return rc;
}

// ===================================================================== ABI

extern "C" {

const char* bc_last_error(void) { return g_last_error.c_str(); }

int bc_get_config(bc_config* out) {
  if (!out) return fail(BC_ERR_INVALID, "null config");
  *out = config_snapshot();
  return BC_OK;
}

int bc_set_config(const bc_config* cfg) {
  if (!cfg) return fail(BC_ERR_INVALID, "null config");
  if (cfg->mode != BC_MODE_BATCHED && cfg->mode != BC_MODE_PLAIN) return fail(BC_ERR_INVALID, "bad mode");
  if (cfg->team_threads && cfg->team_threads != 32 && cfg->team_threads != 128 && cfg->team_threads != 256 &&
      cfg->team_threads != 512 && cfg->team_threads != 1024)
    return fail(BC_ERR_INVALID, "team_threads must be 0, 32, 128, 256, 512 or 1024");
  if (cfg->settle_in > 3) return fail(BC_ERR_INVALID, "settle_in must be 0, 1, 2 or 3");
  if (cfg->algorithm > BC_ALGO_DELTA) return fail(BC_ERR_INVALID, "algorithm must be 0, 1 or 2");
  if (cfg->mem_fraction < 0 || cfg->mem_fraction > 0.95) return fail(BC_ERR_INVALID, "mem_fraction out of range");
  if (cfg->team_degree && cfg->warp_degree && cfg->team_degree < cfg->warp_degree)
    return fail(BC_ERR_INVALID, "team_degree must be >= warp_degree");
  std::lock_guard<std::mutex> lk(g_cfg_mu);
  g_cfg = *cfg;
  return BC_OK;
}

int bc_graph_create(const uint64_t* row_ptr, const uint32_t* col_idx, const uint32_t* w, uint32_t n, uint64_t nnz,
                    uint32_t flags, bc_graph_t* out) {
  if (!out) return fail(BC_ERR_INVALID, "null output handle");
  *out = nullptr;
  if (n == 0) return fail(BC_ERR_INVALID, "n must be >= 1");
  if (n > 0xfffffff0u) return fail(BC_ERR_INVALID, "n too large");
  if (!row_ptr) return fail(BC_ERR_INVALID, "null row_ptr");
  if (nnz >= (1ull << 32)) return fail(BC_ERR_INVALID, "graphs with 2^32 or more CSR entries are not supported");
  if (nnz > 0 && (!col_idx || !w)) return fail(BC_ERR_INVALID, "null col_idx or weights");
  if (row_ptr[0] != 0) return fail(BC_ERR_INVALID, "row_ptr[0] != 0");
  for (uint32_t v = 0; v < n; ++v)
    if (row_ptr[v + 1] < row_ptr[v]) return fail(BC_ERR_INVALID, "row_ptr decreases at %u", v);
  if (row_ptr[n] != nnz) return fail(BC_ERR_INVALID, "row_ptr[n] != nnz");
  uint32_t max_w = 0;
  for (uint64_t e = 0; e < nnz; ++e) {
    if (col_idx[e] >= n) return fail(BC_ERR_INVALID, "col_idx[%llu] = %u out of range", (unsigned long long)e, col_idx[e]);
    if (w[e] == 0) return fail(BC_ERR_INVALID, "weight 0 at entry %llu", (unsigned long long)e);
    max_w = std::max(max_w, w[e]);
  }
  const bool directed = (flags & BC_DIRECTED) != 0;
  if (directed && (flags & BC_UNDIRECTED_CHECK))
    return fail(BC_ERR_INVALID, "BC_DIRECTED and BC_UNDIRECTED_CHECK exclude each other");
  if (flags & BC_UNDIRECTED_CHECK) {
    std::vector<std::array<uint32_t, 3>> a, b;
    a.reserve(nnz);
    b.reserve(nnz);
    for (uint32_t v = 0; v < n; ++v)
      for (uint64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
        a.push_back({v, col_idx[e], w[e]});
        b.push_back({col_idx[e], v, w[e]});
      }
    std::sort(a.begin(), a.end());
    std::sort(b.begin(), b.end());
    if (a != b) return fail(BC_ERR_INVALID, "graph is not symmetric (BC_UNDIRECTED_CHECK)");
  }
  // Layout: optionally renumber vertices by decreasing degree (stable), so
  // the per-source state of the vertices most edges point at is contiguous.
  bool relabel = false;
  // degree used for ordering: out-degree, plus in-degree for directed graphs
  std::vector<uint64_t> tdeg(n);
  for (uint32_t v = 0; v < n; ++v) tdeg[v] = row_ptr[v + 1] - row_ptr[v];
  if (directed)
    for (uint64_t e = 0; e < nnz; ++e) ++tdeg[col_idx[e]];
  if (flags & BC_RELABEL_DEGREE) {
    relabel = true;
  } else if (!(flags & BC_KEEP_ORDER) && n >= 1024) {
    std::vector<uint64_t> degs(tdeg);
    const size_t top = std::max<size_t>(1, n / 100);
    std::nth_element(degs.begin(), degs.begin() + top, degs.end(), std::greater<uint64_t>());
    uint64_t top_sum = 0;
    for (size_t i = 0; i < top; ++i) top_sum += degs[i];
    relabel = nnz > 0 && (double)top_sum > (directed ? 0.20 : 0.10) * (double)nnz;
  }
  std::vector<uint64_t> rp2;
  std::vector<uint32_t> col2, w2, n2o, o2n, e2o;
  if (relabel) {
    n2o.resize(n);
    for (uint32_t v = 0; v < n; ++v) n2o[v] = v;
    std::stable_sort(n2o.begin(), n2o.end(), [&](uint32_t a, uint32_t b) { return tdeg[a] > tdeg[b]; });
    o2n.resize(n);
    for (uint32_t i = 0; i < n; ++i) o2n[n2o[i]] = i;
    rp2.resize((size_t)n + 1);
    col2.resize(nnz);
    w2.resize(nnz);
    e2o.resize(nnz);
    rp2[0] = 0;
    std::vector<std::pair<uint32_t, uint32_t>> row;  // (new neighbour id, old entry)
    for (uint32_t i = 0; i < n; ++i) {
      const uint32_t o = n2o[i];
      const uint64_t deg = row_ptr[o + 1] - row_ptr[o];
      rp2[i + 1] = rp2[i] + deg;
      // each row sorted by new neighbour id: the gathers of one row then walk
      // the per-source arrays in address order
      row.resize(deg);
      for (uint64_t j = 0; j < deg; ++j) {
        const uint64_t eo = row_ptr[o] + j;
        row[j] = {o2n[col_idx[eo]], (uint32_t)eo};
      }
      std::sort(row.begin(), row.end());
      for (uint64_t j = 0; j < deg; ++j) {
        const uint64_t en = rp2[i] + j;
        col2[en] = row[j].first;
        w2[en] = w[row[j].second];
        e2o[en] = row[j].second;
      }
    }
    row_ptr = rp2.data();
    col_idx = col2.data();
    w = w2.data();
  }
  // directed: the in-edge CSR (transpose), each row sorted by source id
  std::vector<uint64_t> irp;
  std::vector<uint32_t> icol, iw;
  if (directed) {
    irp.assign((size_t)n + 1, 0);
    for (uint64_t e = 0; e < nnz; ++e) ++irp[(size_t)col_idx[e] + 1];
    for (uint32_t v = 0; v < n; ++v) irp[v + 1] += irp[v];
    std::vector<uint64_t> fill(irp.begin(), irp.end() - 1);
    icol.resize(nnz);
    iw.resize(nnz);
    for (uint32_t v = 0; v < n; ++v)
      for (uint64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
        const uint64_t pos = fill[col_idx[e]]++;
        icol[pos] = v;
        iw[pos] = w[e];
      }
  }
  auto g = std::make_unique<bc_graph>();
  CK(cudaGetDevice(&g->device));
  CK(cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, g->device));
  g->n = n;
  g->nnz = nnz;
  g->max_w = max_w;
  {
    // default split width: the mean Delta_node (measured against max_w / 4:
    // BA 65k +36%, grid +1%, R-MAT +0.3%, ER 1k -8%)
    double sum = 0.0;
    uint64_t rows = 0;
    for (uint32_t v = 0; v < n; ++v) {
      if (row_ptr[v + 1] == row_ptr[v]) continue;
      uint32_t m = 0xffffffffu;
      for (uint64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) m = std::min(m, w[e]);
      sum += m;
      ++rows;
    }
    g->width_default = rows ? std::max<uint64_t>(1, (uint64_t)(sum / (double)rows + 0.5)) : 1;
  }
  g->dist_bits = distance_bits(n, row_ptr, col_idx, w, max_w, directed);
  g->fingerprint = fingerprint(n, nnz, row_ptr, col_idx, w);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(g->fingerprint);
    if (it != g_tune_cache.end()) g->tuned = it->second;
  }
  uint32_t* d_col = nullptr;
  uint32_t* d_w = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&g->row_ptr, ((size_t)n + 1) * 8);
  // packed adjacency when bits(n - 1) + bits(max weight) <= 32
  uint32_t col_bits = 1, w_bits = 1;
  while (col_bits < 32 && (1ull << col_bits) < (uint64_t)n) ++col_bits;
  while (w_bits < 32 && (1ull << w_bits) <= (uint64_t)max_w) ++w_bits;
  const bool packed = col_bits + w_bits <= 32 && g->dist_bits == 32;
  if (packed) {
    g->col_bits = col_bits;
    if (e == cudaSuccess) e = cudaMalloc(&g->adjp, std::max<size_t>(nnz, 1) * 4);
  } else {
    if (e == cudaSuccess) e = cudaMalloc(&g->adj, std::max<size_t>(nnz, 1) * 8);
  }
  if (e == cudaSuccess) e = cudaMalloc(&g->dnode, (size_t)n * 4);
  if (!directed) {
    if (e == cudaSuccess) e = cudaMalloc(&g->dnode2, (size_t)n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&g->dnode_arg, (size_t)n * 4);
  }
  if (e == cudaSuccess) e = cudaMalloc(&d_col, std::max<size_t>(nnz, 1) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&d_w, std::max<size_t>(nnz, 1) * 4);
  if (e == cudaSuccess) e = cudaMemcpyAsync(g->row_ptr, row_ptr, ((size_t)n + 1) * 8, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(d_col, col_idx, nnz * 4, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(d_w, w, nnz * 4, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess && relabel) {
    g->relabeled = true;
    e = cudaMalloc(&g->o2n, (size_t)n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&g->n2o, (size_t)n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&g->e2o, std::max<size_t>(nnz, 1) * 4);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->o2n, o2n.data(), (size_t)n * 4, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->n2o, n2o.data(), (size_t)n * 4, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(g->e2o, e2o.data(), nnz * 4, cudaMemcpyHostToDevice, g->stream);
    g->h_o2n = o2n;
  }
  if (e == cudaSuccess)
    e = launch_prep(n, nnz, g->row_ptr, d_col, d_w, g->adj, g->dnode, g->dnode2, g->dnode_arg, g->stream);
  if (e == cudaSuccess && packed) e = launch_pack32(nnz, d_col, d_w, col_bits, g->adjp, g->stream);
  if (directed && e == cudaSuccess) {
    // same entry form for the in-edge CSR; d_col / d_w are reused for it
    g->directed = true;
    e = cudaStreamSynchronize(g->stream);
    if (e == cudaSuccess) e = cudaMalloc(&g->in_row_ptr, ((size_t)n + 1) * 8);
    if (e == cudaSuccess) e = cudaMalloc(&g->dnode_in, (size_t)n * 4);
    if (e == cudaSuccess) {
      if (packed) e = cudaMalloc(&g->in_adjp, std::max<size_t>(nnz, 1) * 4);
      else e = cudaMalloc(&g->in_adj, std::max<size_t>(nnz, 1) * 8);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->in_row_ptr, irp.data(), ((size_t)n + 1) * 8, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(d_col, icol.data(), nnz * 4, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(d_w, iw.data(), nnz * 4, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess)
      e = launch_prep(n, nnz, g->in_row_ptr, d_col, d_w, g->in_adj, g->dnode_in, nullptr, nullptr, g->stream);
    if (e == cudaSuccess && packed) e = launch_pack32(nnz, d_col, d_w, col_bits, g->in_adjp, g->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  cudaFree(d_col);
  cudaFree(d_w);
  if (e != cudaSuccess) {
    cudaFree(g->row_ptr);
    cudaFree(g->adj);
    cudaFree(g->adjp);
    cudaFree(g->dnode);
    cudaFree(g->dnode2);
    cudaFree(g->dnode_arg);
    cudaFree(g->o2n);
    cudaFree(g->n2o);
    cudaFree(g->e2o);
    cudaFree(g->in_row_ptr);
    cudaFree(g->in_adj);
    cudaFree(g->in_adjp);
    cudaFree(g->dnode_in);
    if (g->stream) cudaStreamDestroy(g->stream);
    return cuda_fail(e, "bc_graph_create upload");
  }
  g->device_bytes = (((uint64_t)n + 1) * 8 + nnz * (packed ? 4 : 8) + (uint64_t)n * 4) * (directed ? 2 : 1) +
                    (directed ? 0 : 8ull * n) + (relabel ? 8ull * n + 4ull * nnz : 0);
  *out = g.release();
  return BC_OK;
}

int bc_graph_destroy(bc_graph_t g) {
  if (int rc = check_graph(g)) return rc;
  if (g->serving_refs.load() > 0) return fail(BC_ERR_BUSY, "graph still has serving requests");
  if (g->step_refs.load() > 0) return fail(BC_ERR_BUSY, "graph still has step graphs (bc_step_destroy them first)");
  cudaSetDevice(g->device);
  cudaDeviceSynchronize();  // async runs on callers' streams may still use the graph's workspaces
  for (auto& w : g->pool) {
    if (w->done) cudaEventSynchronize(w->done);
    ws_free(w.get());
  }
  g->pool.clear();
  plain_destroy(g->plain);
  paper_destroy(g->paper);
  cudaFree(g->row_ptr);
  cudaFree(g->adj);
  cudaFree(g->adjp);
  cudaFree(g->dnode);
  cudaFree(g->dnode2);
  cudaFree(g->dnode_arg);
  cudaFree(g->ebc);
  cudaFree(g->o2n);
  cudaFree(g->n2o);
  cudaFree(g->e2o);
  cudaFree(g->esm);
  cudaFree(g->in_row_ptr);
  cudaFree(g->in_adj);
  cudaFree(g->in_adjp);
  cudaFree(g->dnode_in);
  cudaStreamDestroy(g->stream);
  delete g;
  return BC_OK;
}

int bc_graph_get_info(bc_graph_t g, bc_graph_info* out) {
  if (int rc = check_graph(g)) return rc;
  if (!out) return fail(BC_ERR_INVALID, "null output");
  out->n = g->n;
  out->nnz = g->nnz;
  out->max_weight = g->max_w;
  out->dist_bits = (uint32_t)g->dist_bits;
  out->device_bytes = g->device_bytes;
  out->slab_bytes = make_layout(g->n, g->dist_bits).stride;
  out->relabeled = g->relabeled ? 1u : 0u;
  out->directed = g->directed ? 1u : 0u;
  return BC_OK;
}

int bc_compute(bc_graph_t g, const uint32_t* sources, uint32_t k, double scale, double* out_bc) {
  if (int rc = check_graph(g)) return rc;
  if (!out_bc) return fail(BC_ERR_INVALID, "null out_bc");
  if (k && !sources) return fail(BC_ERR_INVALID, "null sources");
  CK(cudaSetDevice(g->device));
  RunCfg r = resolve(g);
  if (r.mode == BC_MODE_PLAIN) return compute_plain(g, sources, k, scale, out_bc, r);
  return compute_sync(g, sources, k, scale, out_bc, nullptr, r);
}

}  // extern "C"

namespace {

// Shared body of the async entry points: device sources in, device outputs.
int compute_async(bc_graph* g, const uint32_t* d_sources, uint32_t k, double scale, double* d_out_bc,
                  double* d_out_ebc, void* stream) {
  if (int rc = check_graph(g)) return rc;
  if (!d_out_bc) return fail(BC_ERR_INVALID, "null d_out_bc");
  if (k && !d_sources) return fail(BC_ERR_INVALID, "null d_sources");
  CK(cudaSetDevice(g->device));
  RunCfg r = resolve(g);
  if (r.mode != BC_MODE_BATCHED) return fail(BC_ERR_INVALID, "the async entry points run the batched mode only");
  if (d_out_ebc)
    if (int rc = ensure_edge_map(g)) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the workspace this stream kept from its previous async call: that run
  // and its status copy are ordered before this one on the stream
  Workspace* prev = nullptr;
  {
    std::lock_guard<std::mutex> lk(g->mu);
    auto it = g->async_ws.find(st);
    if (it != g->async_ws.end()) {
      prev = it->second;
      g->async_ws.erase(it);
    }
  }
  if (prev) ws_release(g, prev, st);
  uint32_t slots = 0;
  int rc = plan_slots(g, r, k, &slots);
  if (rc) return rc;
  Workspace* w = nullptr;
  if ((rc = ws_acquire(g, slots, 0, st, &w))) return rc;
  rc = enqueue_batched(g, w, r, d_sources, k, scale, d_out_bc, d_out_ebc, slots, 0, st, true);
  if (!rc) {
    cudaError_t e = cudaMemcpyAsync(w->host_ctl, w->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync(control)");
  }
  if (rc) {
    ws_release(g, w, st);
    return rc;
  }
  // the workspace stays with this stream until bc_sync_status (or the
  // stream's next async call) has read its status block
  std::lock_guard<std::mutex> lk(g->mu);
  g->async_ws[st] = w;
  g->last.algorithm = r.algo == ALGO_DELTA ? BC_ALGO_DELTA : BC_ALGO_STRICT;
  g->last.team_threads = r.team;
  g->last.slots = slots;
  g->last.bucket_width = r.width;
  g->last.warp_degree = r.warp_deg;
  g->last.team_degree = r.team_deg;
  g->last.settle_in = r.settle_in ? (r.refine ? 1u : 3u) : 2u;
  return BC_OK;
}

}  // namespace

extern "C" {

int bc_compute_async(bc_graph_t g, const uint32_t* d_sources, uint32_t k, double scale, double* d_out_bc,
                     void* stream) {
  return compute_async(g, d_sources, k, scale, d_out_bc, nullptr, stream);
}

int bc_edge_compute_async(bc_graph_t g, const uint32_t* d_sources, uint32_t k, double scale, double* d_out_ebc,
                          double* d_out_bc, void* stream) {
  if (!d_out_ebc) return fail(BC_ERR_INVALID, "null d_out_ebc");
  return compute_async(g, d_sources, k, scale, d_out_bc, d_out_ebc, stream);
}

int bc_sync_status(bc_graph_t g, void* stream) {
  if (int rc = check_graph(g)) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CK(cudaSetDevice(g->device));
  const cudaError_t se = cudaStreamSynchronize(st);
  Workspace* w = nullptr;
  {
    std::lock_guard<std::mutex> lk(g->mu);
    auto it = g->async_ws.find(st);
    if (it != g->async_ws.end()) {
      w = it->second;
      g->async_ws.erase(it);
    }
  }
  if (se != cudaSuccess) {
    // the stream's work has ended (with an error): its workspace goes back to the pool
    if (w) ws_release(g, w, st);
    return cuda_fail(se, "cudaStreamSynchronize");
  }
  if (!w) return BC_OK;
  const Ctl c = *w->host_ctl;  // read before the workspace goes back to the pool
  ws_release(g, w, st);
  {
    std::lock_guard<std::mutex> lk(g->mu);
    g->last.sources = c.stats[STAT_SOURCES];
    g->last.phases = c.stats[STAT_PHASES];
    g->last.refills = c.stats[STAT_REFILLS];
    g->last.reached = c.stats[STAT_REACHED];
    g->last.relax_atomics = c.stats[STAT_RELAX];
    g->last.entries_scanned = c.stats[STAT_ENTRIES];
    g->last.dag_edges = c.stats[STAT_DAG_EDGES];
    g->last.pair_overflows = c.stats[STAT_PAIR_OVERFLOW];
    g->last.cycles_expand = c.stats[STAT_CYC_EXPAND];
    g->last.cycles_refill = c.stats[STAT_CYC_REFILL];
    g->last.cycles_settle = c.stats[STAT_CYC_SETTLE];
    g->last.cycles_backward = c.stats[STAT_CYC_BACKWARD];
    g->last.near_scanned = c.stats[STAT_NEAR_SCANNED];
    g->last.far_scanned = c.stats[STAT_FAR_SCANNED];
    g->last.levels = c.stats[STAT_LEVELS];
  }
  return status_from_dev(c.err);
}

int bc_edge_compute(bc_graph_t g, const uint32_t* sources, uint32_t k, double scale, double* out_ebc,
                    double* out_bc) {
  if (int rc = check_graph(g)) return rc;
  if (!out_ebc) return fail(BC_ERR_INVALID, "null out_ebc");
  if (k && !sources) return fail(BC_ERR_INVALID, "null sources");
  CK(cudaSetDevice(g->device));
  RunCfg r = resolve(g);
  std::vector<double> tmp;
  if (!out_bc) {
    tmp.resize(g->n);
    out_bc = tmp.data();
  }
  return compute_sync(g, sources, k, scale, out_bc, out_ebc, r);
}

int bc_sssp_debug(bc_graph_t g, uint32_t s, uint64_t* out_dist, double* out_sigma, uint32_t* out_level) {
  if (int rc = check_graph(g)) return rc;
  if (s >= g->n) return fail(BC_ERR_INVALID, "source out of range");
  CK(cudaSetDevice(g->device));
  RunCfg r = resolve(g);
  cudaStream_t st = g->stream;
  Workspace* w = nullptr;
  int rc = ws_acquire(g, 1, 1, st, &w);
  if (rc) return rc;
  w->host_src[0] = s;  // the kernel maps caller ids to internal ids
  const uint32_t n = g->n;
  std::vector<uint8_t> dbuf((size_t)n * (g->dist_bits / 8));
  std::vector<double> sig(n);
  std::vector<uint32_t> S(n), ends((size_t)n + 2);
  cudaError_t e = cudaMemcpyAsync(w->src, w->host_src, 4, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    ws_release(g, w, st);
    return cuda_fail(e, "cudaMemcpyAsync");
  }
  rc = enqueue_batched(g, w, r, w->src, 1, 1.0, nullptr, nullptr, 1, RUN_FORWARD_ONLY, st, false);
  if (rc) {
    ws_release(g, w, st);
    return rc;
  }
  char* base = w->slabs;
  e = cudaMemcpyAsync(w->host_ctl, w->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dbuf.data(), base + w->lay.off_d, dbuf.size(), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sig.data(), base + w->lay.off_sig, (size_t)n * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S.data(), base + w->lay.off_S, (size_t)n * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ends.data(), base + w->lay.off_ends, ((size_t)n + 2) * 4, cudaMemcpyDeviceToHost, st);
  // restore the slab invariant (forward-only runs leave distances behind)
  if (e == cudaSuccess) e = cudaMemsetAsync(base + w->lay.off_d, 0xff, dbuf.size(), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  const Ctl c = *w->host_ctl;  // read before the workspace goes back to the pool
  ws_release(g, w, st);
  if (e != cudaSuccess) return cuda_fail(e, "bc_sssp_debug");
  if ((rc = status_from_dev(c.err))) return rc;
  const uint32_t nlev = c.debug[0];
  const uint32_t reached = c.debug[1];
  std::vector<uint32_t> level(n, 0xffffffffu);
  for (uint32_t l = 0; l < nlev; ++l)
    for (uint32_t i = ends[l]; i < ends[l + 1] && i < reached; ++i) level[S[i]] = l;
  for (uint32_t ov = 0; ov < n; ++ov) {
    const uint32_t v = g->relabeled ? g->h_o2n[ov] : ov;  // internal id
    const bool reached_v = level[v] != 0xffffffffu;
    if (out_dist) {
      if (!reached_v) out_dist[ov] = UINT64_MAX;
      else if (g->dist_bits == 32) out_dist[ov] = reinterpret_cast<const uint32_t*>(dbuf.data())[v];
      else out_dist[ov] = reinterpret_cast<const uint64_t*>(dbuf.data())[v];
    }
    if (out_sigma) out_sigma[ov] = reached_v ? sig[v] : 0.0;
    if (out_level) out_level[ov] = level[v];
  }
  return BC_OK;
}

int bc_compute_paper_variant(bc_graph_t g, const uint32_t* sources, uint32_t k, double scale, double* out_bc,
                             int node_parallel, int vwarp) {
  if (int rc = check_graph(g)) return rc;
  if (!out_bc || (k && !sources)) return fail(BC_ERR_INVALID, "null argument");
  if (vwarp != 1 && vwarp != 4 && vwarp != 8 && vwarp != 16 && vwarp != 32)
    return fail(BC_ERR_INVALID, "vwarp must be 1, 4, 8, 16 or 32");
  if (g->directed) return fail(BC_ERR_INVALID, "the paper's mappings run undirected graphs only");
  for (uint32_t i = 0; i < k; ++i)
    if (sources[i] >= g->n) return fail(BC_ERR_INVALID, "source %u out of range (n = %u)", sources[i], g->n);
  CK(cudaSetDevice(g->device));
  RunCfg r = resolve(g);
  cudaStream_t st = g->stream;
  if (!g->paper) {
    cudaError_t e;
    g->paper = paper_create(g->n, g->dist_bits, &e);
    if (!g->paper) return cuda_fail(e, "paper-variant workspace");
  }
  double* d_bc = nullptr;
  CK(cudaMalloc(&d_bc, (size_t)g->n * 8));
  cudaError_t e = cudaMemsetAsync(d_bc, 0, (size_t)g->n * 8, st);
  int dev = DEV_OK;
  unsigned long long stats[STAT_COUNT] = {0};
  if (e == cudaSuccess)
    e = paper_run(g->paper, view(g), g->dist_bits, sources, g->relabeled ? g->h_o2n.data() : nullptr, k, d_bc,
                  node_parallel != 0, vwarp, r.phase_cap, g->sm_count, st, &dev, stats);
  if (e == cudaSuccess && scale != 1.0) e = launch_scale(d_bc, g->n, scale, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_bc, d_bc, (size_t)g->n * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d_bc);
  if (e != cudaSuccess) return cuda_fail(e, "paper-variant run");
  Ctl c{};
  memcpy(c.stats, stats, sizeof stats);
  record_stats(g, c, r, 1);
  return status_from_dev(dev);
}

int bc_last_run_stats(bc_graph_t g, bc_run_stats* out) {
  if (int rc = check_graph(g)) return rc;
  if (!out) return fail(BC_ERR_INVALID, "null output");
  std::lock_guard<std::mutex> lk(g->mu);
  *out = g->last;
  return BC_OK;
}

int bc_autotune(bc_graph_t g, const uint32_t* sources, uint32_t k_probe) {
  if (int rc = check_graph(g)) return rc;
  if (!sources || k_probe == 0) return fail(BC_ERR_INVALID, "autotune needs probe sources");
  CK(cudaSetDevice(g->device));
  bc_config user = config_snapshot();
  // candidates: team size x near/far split width, then sources in flight
  std::vector<uint32_t> teams = {128, 256, 512};
  if (g->dist_bits == 32) teams.push_back(1024);
  std::vector<uint64_t> widths;
  for (uint64_t d : {16ull, 4ull, 1ull}) {
    const uint64_t wv = std::max<uint64_t>(1, g->max_w / d);
    if (std::find(widths.begin(), widths.end(), wv) == widths.end()) widths.push_back(wv);
  }
  std::vector<double> out(g->n);
  auto timed = [&](const RunCfg& r, double* ms) -> int {
    auto t0 = std::chrono::steady_clock::now();
    int rc = compute_sync(g, sources, k_probe, 1.0, out.data(), nullptr, r);
    *ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return rc;
  };
  RunCfg base = resolve(g);
  base.mode = BC_MODE_BATCHED;
  base.settle_in = 1;
  base.refine = (g->dnode2 && user.settle_in == 1) ? 1u : 0u;
  base.algo = (user.algorithm == BC_ALGO_DELTA) ? ALGO_DELTA : ALGO_STRICT;
  // every candidate starts from the built-in thresholds (not a previous tuning)
  base.warp_deg = user.warp_degree ? user.warp_degree : 32u;
  auto team_deg_of = [&](uint32_t team, uint32_t warp_deg) {
    return std::max(user.team_degree ? user.team_degree : 8u * team, warp_deg);
  };
  base.team_deg = team_deg_of(base.team, base.warp_deg);
  double ms = 0;
  if (int rc = timed(base, &ms)) return rc;  // warm-up: workspace allocation
  double best_ms = 1e300;
  double best_phases = 0;  // settle phases per source of the fastest strict candidate
  TuneCfg best;
  for (uint32_t team : teams) {
    if (user.team_threads && user.team_threads != team) continue;
    if (user.algorithm == BC_ALGO_DELTA) break;
    for (uint64_t width : widths) {
      if (user.bucket_width && user.bucket_width != width) continue;
      RunCfg r = base;
      r.team = team;
      r.width = width;
      r.team_deg = team_deg_of(team, r.warp_deg);
      if (int rc = timed(r, &ms)) return rc;
      if (ms < best_ms) {
        best_ms = ms;
        best.team = team;
        best.width = width;
        best.settle_in = 3;
        best.algo = BC_ALGO_STRICT;
        std::lock_guard<std::mutex> lk(g->mu);
        best_phases = g->last.sources ? (double)g->last.phases / (double)g->last.sources : 0.0;
      }
    }
  }
  // the delta-stepping schedule, buckets one to sixteen maximum weights wide:
  // it walks every reached row about four times (rounds, predecessor count,
  // sigma push, backward) against about once, so it is only a candidate where
  // the strict schedule needs many settle phases per source (high diameter)
  if (user.algorithm == BC_ALGO_DELTA || (user.algorithm == BC_ALGO_AUTO && best_phases >= 1000.0)) {
    for (uint32_t team : teams) {
      if (user.team_threads && user.team_threads != team) continue;
      if (!user.team_threads && best.team && team != best.team) continue;
      for (uint64_t m : {1ull, 4ull, 16ull}) {
        const uint64_t width = std::max<uint64_t>(1, g->max_w) * m;
        if (user.bucket_width && user.bucket_width != width) continue;
        RunCfg r = base;
        r.algo = ALGO_DELTA;
        r.team = team;
        r.width = width;
        r.team_deg = team_deg_of(team, r.warp_deg);
        if (int rc = timed(r, &ms)) return rc;
        if (ms < best_ms) {
          best_ms = ms;
          best.team = team;
          best.width = width;
          best.settle_in = 3;
          best.algo = BC_ALGO_DELTA;
        }
      }
    }
  }
  if (best.team == 0) return fail(BC_ERR_INVALID, "autotune: the configuration pins every candidate out");
  // degree thresholds of the strict schedule's expansion tiers: first the
  // warp threshold, then the team threshold (as a multiple of the team size)
  if (best.algo == BC_ALGO_STRICT) {
    RunCfg r = base;
    r.team = best.team;
    r.width = best.width;
    if (!user.warp_degree) {
      uint32_t best_wd = r.warp_deg;
      for (uint32_t wd : {8u, 16u, 32u, 64u}) {
        if (wd == r.warp_deg) continue;  // the built-in value was timed with the team and width above
        r.warp_deg = wd;
        r.team_deg = team_deg_of(r.team, wd);
        if (int rc = timed(r, &ms)) return rc;
        if (ms < best_ms) {
          best_ms = ms;
          best_wd = wd;
        }
      }
      r.warp_deg = best_wd;
      r.team_deg = team_deg_of(r.team, best_wd);
      best.warp_deg = best_wd;
    }
    if (!user.team_degree) {
      uint32_t best_td = 0;
      for (uint32_t mult : {2u, 32u}) {
        r.team_deg = std::max(mult * r.team, r.warp_deg);
        if (int rc = timed(r, &ms)) return rc;
        if (ms < best_ms) {
          best_ms = ms;
          best_td = r.team_deg;
        }
      }
      if (best_td) best.team_deg = best_td;
    }
  }
  // the settle test with the settled-neighbour refinement of Delta_node:
  // fewer, larger batches (high-diameter graphs) against one more gather per
  // candidate and settle pass (dense graphs)
  if (best.algo == BC_ALGO_STRICT && !user.settle_in) best.settle_in = 3;
  if (!user.settle_in && g->dnode2 && best.algo == BC_ALGO_STRICT) {
    RunCfg r = base;
    r.team = best.team;
    r.width = best.width;
    if (best.warp_deg) r.warp_deg = best.warp_deg;
    r.team_deg = best.team_deg ? best.team_deg : team_deg_of(r.team, r.warp_deg);
    r.refine = 1;
    if (int rc = timed(r, &ms)) return rc;
    if (ms < best_ms) {
      best_ms = ms;
      best.settle_in = 1;
    }
  }
  // sources in flight: the full resident capacity, or half of it
  if (!user.max_slots) {
    RunCfg r = base;
    r.team = best.team;
    r.width = best.width;
    r.algo = best.algo == BC_ALGO_DELTA ? ALGO_DELTA : ALGO_STRICT;
    if (best.warp_deg) r.warp_deg = best.warp_deg;
    r.team_deg = best.team_deg ? best.team_deg : team_deg_of(r.team, r.warp_deg);
    r.refine = best.settle_in == 1 ? 1u : 0u;
    uint32_t full = 0;
    if (int rc = plan_slots(g, r, k_probe, &full)) return rc;
    r.max_slots = std::max<uint32_t>(1, full / 2);
    if (int rc = timed(r, &ms)) return rc;
    if (ms < best_ms) {
      best_ms = ms;
      best.max_slots = r.max_slots;
    }
  }
  g->tuned = best;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[g->fingerprint] = best;
  return BC_OK;
}

// ---- step graphs --------------------------------------------------------

}  // extern "C"

struct bc_step {
  bc_graph* g = nullptr;
  Workspace ws;  // private: never in the graph's pool
  RunCfg r{};
  uint32_t slots = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

void step_free(bc_step* s) {
  if (s->exec) cudaGraphExecDestroy(s->exec);
  if (s->graph) cudaGraphDestroy(s->graph);
  ws_free(&s->ws);
}

}  // namespace

extern "C" {

int bc_step_create(bc_graph_t g, const uint32_t* d_sources, uint32_t k, double scale, double* d_out_bc,
                   bc_step_t* out) {
  if (!out) return fail(BC_ERR_INVALID, "null output handle");
  *out = nullptr;
  if (int rc = check_graph(g)) return rc;
  if (!d_out_bc) return fail(BC_ERR_INVALID, "null d_out_bc");
  if (k && !d_sources) return fail(BC_ERR_INVALID, "null d_sources");
  CK(cudaSetDevice(g->device));
  RunCfg r = resolve(g);
  if (r.mode != BC_MODE_BATCHED) return fail(BC_ERR_INVALID, "step graphs capture the batched mode only");
  auto s = std::make_unique<bc_step>();
  s->g = g;
  s->r = r;
  if (int rc = plan_slots(g, r, k, &s->slots)) return rc;
  Workspace& w = s->ws;
  w.slots = s->slots;
  w.lay = make_layout(g->n, g->dist_bits);
  w.bytes = w.lay.stride * s->slots;
  cudaStream_t cap = nullptr;
  cudaError_t e = cudaMalloc(&w.slabs, w.bytes);
  if (e == cudaSuccess) e = cudaMalloc(&w.ctl, sizeof(Ctl));
  if (e == cudaSuccess) e = cudaMallocHost(&w.host_ctl, sizeof(Ctl));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  // the slab invariant, established once: later runs restore it themselves
  if (e == cudaSuccess)
    e = launch_fill_slabs(w.slabs, w.lay.stride, s->slots, w.lay.off_d,
                          align256((uint64_t)g->n * (g->dist_bits / 8)), 0xffffffffu, cap);
  if (e == cudaSuccess)
    e = launch_fill_slabs(w.slabs, w.lay.stride, s->slots, w.lay.off_acc, align256((uint64_t)g->n * 8), 0u, cap);
  if (e == cudaSuccess)
    e = launch_fill_slabs(w.slabs, w.lay.stride, s->slots, w.lay.off_pc, align256((uint64_t)g->n * 4), 0u, cap);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cap);
  if (e != cudaSuccess) {
    if (cap) cudaStreamDestroy(cap);
    step_free(s.get());
    return cuda_fail(e, "step workspace");
  }
  // capture: zero control block and output, source check, persistent kernel,
  // scale, status copy to pinned host memory
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  int rc = BC_OK;
  if (e == cudaSuccess) {
    rc = enqueue_batched(g, &w, r, d_sources, k, scale, d_out_bc, nullptr, s->slots, 0, cap, true);
    if (!rc) {
      cudaError_t e2 = cudaMemcpyAsync(w.host_ctl, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, cap);
      if (e2 != cudaSuccess) rc = cuda_fail(e2, "cudaMemcpyAsync(control) during capture");
    }
    e = cudaStreamEndCapture(cap, &s->graph);  // always end the capture, also after a failed enqueue
  }
  if (e == cudaSuccess && !rc) e = cudaGraphInstantiate(&s->exec, s->graph, 0);
  cudaStreamDestroy(cap);
  if (rc || e != cudaSuccess) {
    step_free(s.get());
    return rc ? rc : cuda_fail(e, "step graph capture");
  }
  g->step_refs += 1;
  *out = s.release();
  return BC_OK;
}

int bc_step_launch(bc_step_t s, void* stream) {
  if (!s) return fail(BC_ERR_INVALID, "null step handle");
  CK(cudaSetDevice(s->g->device));
  CK(cudaGraphLaunch(s->exec, static_cast<cudaStream_t>(stream)));
  return BC_OK;
}

int bc_step_sync(bc_step_t s, void* stream) {
  if (!s) return fail(BC_ERR_INVALID, "null step handle");
  CK(cudaSetDevice(s->g->device));
  CK(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  record_stats(s->g, *s->ws.host_ctl, s->r, s->slots);
  return status_from_dev(s->ws.host_ctl->err);
}

int bc_step_destroy(bc_step_t s) {
  if (!s) return fail(BC_ERR_INVALID, "null step handle");
  cudaSetDevice(s->g->device);
  cudaDeviceSynchronize();  // no launch of this step may still be in flight
  s->g->step_refs -= 1;
  step_free(s);
  delete s;
  return BC_OK;
}

}  // extern "C"
