// Internal declarations shared by the CUDA translation units of libbcgpu.
// Not part of the public ABI (that is include/bcgpu.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace bcgpu {

// Graph as the kernels see it (Sec. 3.1: CSR plus a parallel weight array,
// here interleaved as one 8-byte {col, w} record per entry).
struct GraphDev {
  uint32_t n;
  uint64_t nnz;
  const uint64_t* row_ptr;  // [n + 1]
  const uint2* adj;         // [nnz] {neighbour, weight}, or nullptr when adjp is used
  const uint32_t* adjp;     // [nnz] neighbour | weight << col_bits (graphs where both fit 32 bits)
  uint32_t col_bits;        // bits of the neighbour id in an adjp word
  const uint32_t* dnode;    // [n] Delta_node(v) = min incident (directed: outgoing) weight, UINT32_MAX if none
  // Undirected graphs (nullptr otherwise): the second smallest incident weight
  // (UINT32_MAX below two entries) and the neighbour of the smallest one
  // (UINT32_MAX if none): once that neighbour is settled, every edge from v to
  // a vertex still unsettled weighs at least dnode2[v].
  const uint32_t* dnode2;
  const uint32_t* dnode_arg;
  // Directed graphs only (nullptr otherwise): the in-edge CSR, same entry
  // form as the out-edge one, and the minimum incoming weight per vertex.
  const uint64_t* in_row_ptr;
  const uint2* in_adj;
  const uint32_t* in_adjp;
  const uint32_t* dnode_in;
  // Optional relabeling (graph prep orders vertices by decreasing degree so
  // the state of high-degree vertices is contiguous).  Internal ids are
  // "new"; the caller's ids are "old".  All three are nullptr when the graph
  // keeps the caller's order.
  const uint32_t* o2n;      // [n] old id -> new id (applied to sources)
  const uint32_t* n2o;      // [n] new id -> old id (applied to BC output)
  const uint32_t* e2o;      // [nnz] new CSR entry -> old CSR entry (edge BC output)
};

// Byte offsets of the per-source arrays inside one slab (one slab per source
// in flight).  d: distances (all INF between sources), sig: sigma during the
// forward pass and the coefficient c = (1 + delta) / sigma during the backward
// pass, S: settle order (the level lists of Algorithm 1's S/ends), ends: level
// boundaries, nearq / farq / farq2: candidate queues (reached, unsettled
// vertices below the split, between the split and split2, above split2).
// acc: per-vertex sum of successor coefficients during the backward pass
// (zero between sources); pend: end of each level's range in the DAG edge
// list; pairs: the shortest-path DAG edges (u -> v) found while pulling sigma,
// in level order of v (capacity pair_cap; on overflow the backward pass falls
// back to scanning every CSR entry); pc: per-vertex round stamps, then
// predecessor counts, of the delta-stepping schedule (zero between sources).
struct SlabLayout {
  uint64_t stride;
  uint64_t off_d, off_sig, off_S, off_ends, off_near, off_far, off_far2, off_acc, off_pend, off_pairs, off_pc;
  uint64_t off_pair_e;  // entry walked by each DAG edge (edge output); 0 = not in this layout
  uint32_t pair_cap;
};

enum : uint32_t {
  RUN_FORWARD_ONLY = 1u,  // stop after distances / sigma / levels (test hook)
};

// Per-source schedules of the batched kernel.
enum : uint32_t {
  ALGO_STRICT = 1,  // strict settle batches (Sec. 3.2), sigma pulled per batch
  ALGO_DELTA = 2,   // delta-stepping distances, then sigma and delta over DAG hop levels
};

enum : int {
  DEV_OK = 0,
  DEV_ERR_INVALID = 1,  // out-of-range source
  DEV_ERR_TIMEOUT = 4,  // phase cap hit
  DEV_ERR_INTERNAL = 5, // a consistency check failed (reported as BC_ERR_CUDA)
};

// Per-run counters (summed over sources).
enum : int {
  STAT_SOURCES = 0,
  STAT_PHASES,
  STAT_REFILLS,
  STAT_REACHED,
  STAT_RELAX,
  STAT_ENTRIES,
  STAT_DAG_EDGES,
  STAT_PAIR_OVERFLOW,
  STAT_CYC_EXPAND,    // SM clock cycles (team leader) spent per section
  STAT_CYC_REFILL,
  STAT_CYC_SETTLE,
  STAT_CYC_BACKWARD,
  STAT_NEAR_SCANNED,  // near / far queue entries read by the threshold, settle and refill passes
  STAT_FAR_SCANNED,
  STAT_LEVELS,        // levels of the backward pass
  STAT_COUNT
};

struct BatchArgs {
  GraphDev g;
  const uint32_t* sources;
  uint32_t k;
  uint32_t* counter;  // [0]: next source index (zeroed before launch)
  double* bc;         // [n] raw sum of delta (scale applied afterwards)
  double* ebc;        // [nnz] raw per-entry shares, or nullptr
  const uint32_t* esm; // edge output with the DAG edge list: walked entry -> output entry, or nullptr
  char* slabs;
  SlabLayout lay;
  uint32_t nslots;
  uint64_t width;      // near/far split width
  uint32_t settle_in;  // apply the strict IN criterion too
  uint32_t refine;     // bound each candidate's edges to unsettled vertices by dnode2 once dnode_arg is settled
  uint64_t phase_cap;  // cap on phases + refills per source
  int* err;            // DEV_* status word
  unsigned long long* stats;  // [STAT_COUNT] or nullptr
  uint32_t warp_deg;   // forward expansion: rows with >= warp_deg entries get a warp each
  uint32_t team_deg;   // ... and rows with >= team_deg entries the whole team
  uint32_t hot_n;      // ids below hot_n are gathered with an L2 evict-last hint
  uint32_t algo;       // ALGO_*
  uint32_t flags;      // RUN_*
  uint32_t* debug_out; // RUN_FORWARD_ONLY: [0] = levels, [1] = reached
};

// Launchers (bc_batched.cu).  team: 32, 128, 256 or 512 threads per source.
cudaError_t launch_batched(const BatchArgs& a, int dist_bits, int team, int grid, cudaStream_t st);
int batched_block_threads(int team);
cudaError_t batched_occupancy(int dist_bits, int team, int* blocks_per_sm);  // strict schedule
cudaError_t batched_occupancy(int dist_bits, int team, int algo, int* blocks_per_sm);
cudaError_t launch_batched_delta(const BatchArgs& a, int dist_bits, int team, int grid, cudaStream_t st);
cudaError_t batched_occupancy_delta(int dist_bits, int team, int* blocks_per_sm);

// Graph preparation and small helpers (bc_prep.cu).
// dnode2 / dnode_arg may be nullptr (not computed).
cudaError_t launch_prep(uint32_t n, uint64_t nnz, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* w,
                        uint2* adj, uint32_t* dnode, uint32_t* dnode2, uint32_t* dnode_arg, cudaStream_t st);
// Packed form: adjp[e] = col[e] | w[e] << col_bits (caller checked that both fit).
cudaError_t launch_pack32(uint64_t nnz, const uint32_t* col, const uint32_t* w, uint32_t col_bits, uint32_t* adjp,
                          cudaStream_t st);
cudaError_t launch_fill_u64(uint64_t* p, uint64_t count, uint64_t value, cudaStream_t st);
cudaError_t launch_scale(double* p, uint64_t count, double scale, cudaStream_t st);
cudaError_t launch_check_sources(const uint32_t* src, uint32_t k, uint32_t n, int* err, cudaStream_t st);
// Fill `bytes` (a multiple of 4) at offset `off` of every slot of a slab array.
cudaError_t launch_fill_slabs(char* base, uint64_t stride, uint32_t nslots, uint64_t off, uint64_t bytes,
                              uint32_t value, cudaStream_t st);

// Record a message for bc_last_error() on the calling thread; returns code.
int set_error(int code, const char* msg);

// The paper's thread mappings (bc_paper.cu): node-parallel or work-efficient
// expansion with VW threads per vertex, Delta_i and settle over all V.
struct PaperWork {
  uint32_t n = 0;
  void* d = nullptr;
  double* sig = nullptr;
  uint32_t* S = nullptr;
  uint8_t* U = nullptr;
  uint8_t* F = nullptr;
  void* ctr = nullptr;
  void* host_ctr = nullptr;  // pinned
};
PaperWork* paper_create(uint32_t n, int dist_bits, cudaError_t* e);
void paper_destroy(PaperWork* w);
uint64_t paper_bytes(uint32_t n, int dist_bits);
cudaError_t paper_run(PaperWork* w, const GraphDev& g, int dist_bits, const uint32_t* host_sources,
                      const uint32_t* host_o2n, uint32_t k, double* bc, bool node_parallel, int vwarp,
                      uint64_t phase_cap, int sm_count, cudaStream_t st, int* status, unsigned long long* stats);

}  // namespace bcgpu

struct bc_graph;

namespace bcgpu {

// Serving support (implemented in bc_api.cu, used by the scheduler in
// bc_serve.cu).  A lease is one request's workspace (slabs, source list,
// device accumulator), held from serve_open to serve_finish; the request's
// sources run as a sequence of source batches (serve_batch), each one
// persistent launch that adds into the accumulator, on whichever stream the
// scheduler picks.  The last batch also scales the sum and copies it to
// pinned host memory; serve_finish hands it to the caller and releases the
// workspace.
struct ServeLease;
struct ServePlan {
  uint32_t team;        // threads per source
  uint32_t max_slots;   // sources the GPU holds at once for this team size
  uint64_t slot_bytes;  // device bytes per source in flight
  uint64_t fixed_bytes; // per-request device bytes besides the slabs
};
int serve_plan(bc_graph* g, ServePlan* out);
// Reserve a workspace of up to slot_cap slabs and stage the sources (on st).
int serve_open(bc_graph* g, const uint32_t* sources, uint32_t k, uint32_t slot_cap, cudaStream_t st,
               ServeLease** out);
uint32_t serve_slot_cap(const ServeLease* l);  // slabs actually held
// Enqueue sources [first, first + count) with `slots` of them in flight; the
// last batch also applies `scale` and stages the result for serve_finish.
int serve_batch(ServeLease* l, uint32_t first, uint32_t count, uint32_t slots, bool last, double scale,
                cudaStream_t st);
bool serve_ready(ServeLease* l);         // the latest batch has completed
int serve_batch_status(ServeLease* l);   // its device status (waits for it)
int serve_finish(ServeLease* l, double* out_bc);  // out_bc may be null (failed request); releases the lease
int graph_device(const bc_graph* g);
uint32_t graph_n(const bc_graph* g);
uint64_t graph_nnz(const bc_graph* g);
void graph_serving_ref(bc_graph* g, int delta);

// Plain form (bc_plain.cu): one source at a time over the whole GPU.
struct PlainWork;
PlainWork* plain_create(uint32_t n, int dist_bits, cudaError_t* e);
void plain_destroy(PlainWork* w);
uint64_t plain_bytes(uint32_t n, int dist_bits);
// Runs sources[0..k) (HOST list) one after another; adds raw delta into bc.
// Returns DEV_* status through *dev_status.
// host_o2n: the graph's old -> new id map on the host (nullptr: no relabeling).
cudaError_t plain_run(PlainWork* w, const GraphDev& g, int dist_bits, const uint32_t* host_sources,
                      const uint32_t* host_o2n, uint32_t k, double* bc, uint64_t width, uint32_t settle_in,
                      uint64_t phase_cap, int sm_count, cudaStream_t st, int* dev_status,
                      unsigned long long* host_stats);

}  // namespace bcgpu
