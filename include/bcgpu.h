/*
 * bcgpu.h - weighted betweenness centrality on one GB300 (sm_103a), C ABI.
 *
 * Method: arxiv 1701.05975, "A GPU-Based Solution to Fast Calculation of
 * Betweenness Centrality on Large Weighted Networks".  For every source s in a
 * caller-given list the library runs Brandes' algorithm (Sec. 2.1): exact
 * single-source shortest paths over the weighted CSR graph with the strict
 * settle criterion of Sec. 3.2 (Eq. 2 with Eq. 4), the shortest-path counts
 * sigma over the resulting DAG, and the backward dependency accumulation
 * delta (Algorithm 3) summed into per-vertex BC.
 *
 * Result convention:  out_bc[v] = scale * sum_{s in sources} delta_s(v),
 *   delta_s(v) = sum_{t != s, v} sigma_st(v) / sigma_st          (Eq. 1 terms).
 * With sources = V and scale = 1 this is Eq. 1 over ordered pairs; pass
 * scale = 0.5 for the usual undirected value, 0.5 * n / k when the k sources
 * are a uniform sample.  Duplicate sources count twice.
 *
 * Graph convention (Sec. 3.1): CSR row_ptr (n + 1 entries, row_ptr[0] = 0,
 * non-decreasing, row_ptr[n] = nnz), col_idx (nnz entries < n) and a parallel
 * weight array (nnz entries, each >= 1).  The graph is undirected (Sec. 2.1):
 * each edge {u, v, w} must be stored as both (u -> v, w) and (v -> u, w).
 * Every CSR entry is a distinct edge: parallel equal-weight entries each count
 * as a shortest path; self-loops are allowed and never lie on a shortest path.
 * A weight of 0 is rejected (the strict criterion of Eq. 4 can stall on it).
 *
 * Numbers: distances are exact integers (uint64 on the ABI; the device keeps
 * uint32 when n * max_weight * 2 < 2^32, else uint64), sigma, delta and BC
 * are IEEE double.
 *
 * Errors: every function returns BC_OK (0) or one of the BC_ERR_* codes
 * below; no C++ exception crosses the ABI.  bc_last_error() returns a
 * thread-local message for the last failing call on the calling thread.
 *
 * Threads: all functions are thread-safe.  All device work runs on the
 * current CUDA device of the calling thread at bc_graph_create time.
 */
#ifndef BCGPU_H
#define BCGPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define BC_OK 0
#define BC_ERR_INVALID 1   /* malformed CSR, weight 0, source >= n, bad handle or argument */
#define BC_ERR_NOMEM 2     /* device or host allocation failed, or the request exceeds the memory budget */
#define BC_ERR_CUDA 3      /* a CUDA runtime call failed (message in bc_last_error) */
#define BC_ERR_TIMEOUT 4   /* a device loop hit its iteration cap, or a wait timed out */
#define BC_ERR_BUSY 5      /* the serving queue is full */
#define BC_ERR_CANCELLED 6 /* the request was cancelled */

/* ---- graph flags ------------------------------------------------------- */
#define BC_UNDIRECTED_CHECK 0x1u /* verify that every (u -> v, w) entry has a (v -> u, w) twin */
#define BC_RELABEL_DEGREE 0x2u   /* always store vertices internally in decreasing-degree order */
#define BC_KEEP_ORDER 0x4u       /* never relabel (default: relabel when the top 1% of vertices by degree
                                    hold more than 10% of the CSR entries) */
#define BC_DIRECTED 0x8u         /* the CSR rows are out-edges of a directed graph (Sec. 2.1: the method
                                    extends to directed graphs); no symmetry is assumed.  Distances and
                                    sigma follow out-edges; BC counts ordered pairs (use scale 1).  The
                                    batched path only (BC_MODE_PLAIN and bc_compute_noalloc are undirected). */

/* ---- execution modes --------------------------------------------------- */
#define BC_MODE_BATCHED 0u /* persistent launch: one team (warp or CTA) per source, many sources in flight */
#define BC_MODE_PLAIN 1u   /* one source at a time over the whole GPU, host-driven phase loop */

/* ---- per-source schedules of the batched mode --------------------------- */
#define BC_ALGO_AUTO 0u   /* the graph's tuned schedule, else BC_ALGO_STRICT */
#define BC_ALGO_STRICT 1u /* the paper's phases: settle every vertex that meets the strict OUT (Eq. 2 + Eq. 4) or
                             IN criterion, sigma pulled as each batch settles (Sec. 3.2, Algorithm 2) */
#define BC_ALGO_DELTA 2u  /* distances by delta-stepping rounds (bucket width = bucket_width), then predecessor
                             counts, sigma pushed down the shortest-path DAG in hop-depth levels, and the
                             dependency pull of Algorithm 3 over those levels in reverse.  Same results; far
                             fewer synchronised steps on high-diameter graphs. */

/* ---- request states (bc_request_poll) ---------------------------------- */
#define BC_REQ_QUEUED 0
#define BC_REQ_RUNNING 1
#define BC_REQ_DONE 2
#define BC_REQ_FAILED 3
#define BC_REQ_CANCELLED 4

typedef struct bc_graph *bc_graph_t;
typedef uint64_t bc_request_t;

/*
 * Tuning and test knobs (process-wide).  A zero field means "automatic":
 * the autotuner (bc_autotune) or the built-in defaults choose it.
 */
typedef struct bc_config {
  uint32_t mode;          /* BC_MODE_BATCHED or BC_MODE_PLAIN */
  uint32_t team_threads;  /* threads that share one source: 32 (warp team) or 128/256/512/1024 (CTA team);
                             1024 needs 32-bit distances and falls back to 512 otherwise.  0 = tuned value,
                             else by entries walked per vertex (>= 20: 1024 or 512, >= 6: 256, else 128) */
  uint32_t max_slots;     /* cap on sources in flight at once (per-source slabs held in device memory) */
  uint32_t settle_in;     /* 1: settle by the strict OUT criterion (Eq. 2 + Eq. 4) OR the strict IN
                             criterion, each with Delta_node raised to the second smallest incident
                             weight once the vertex's lightest neighbour is known to be settled
                             (undirected graphs; a legal refinement, larger batches); 2: OUT only with
                             Delta_node (the paper's criterion alone); 3: OUT or IN with Delta_node;
                             0 = automatic (tuned, else 3) */
  uint64_t bucket_width;  /* near/far split width, in distance units (>= 1); 0 = tuned value, else the
                             mean over non-empty rows of the row's smallest weight (Delta_node) */
  uint64_t phase_cap;     /* device cap on phases + queue refills per source; hitting it returns BC_ERR_TIMEOUT.
                             0 = automatic: 4n + 64, above what any valid input needs (phases <= n,
                             refills <= 3n + 2) */
  double mem_fraction;    /* share of free device memory the slabs may take (0 < f <= 0.95); 0 = 0.6 */
  uint32_t warp_degree;   /* forward expansion: rows with at least this many entries get one warp each
                             (0 = 32) */
  uint32_t team_degree;   /* ... and rows with at least this many entries the whole team (>= warp_degree;
                             0 = 8 x team_threads) */
  uint32_t algorithm;     /* BC_ALGO_AUTO, BC_ALGO_STRICT or BC_ALGO_DELTA (batched mode) */
  uint32_t hot_vertices;  /* on degree-relabeled graphs, the distance words of this many leading (highest-
                             degree) vertex ids are gathered with an L2 evict-last hint; 0 = 32768 */
} bc_config;

/* Read the current process-wide configuration. */
int bc_get_config(bc_config *out);

/* Replace the process-wide configuration (validated; BC_ERR_INVALID on a bad field). */
int bc_set_config(const bc_config *cfg);

/* Thread-local description of the last error on this thread ("" if none). */
const char *bc_last_error(void);

/*
 * Upload a graph (Sec. 3.1 CSR + weight array) to the current device.
 * row_ptr[n + 1], col_idx[nnz] and w[nnz] are HOST arrays; the library copies
 * them and the caller keeps ownership.  Limits: 1 <= n <= 0xFFFFFFF0 and nnz < 2^32
 * (checked before any array is read).  Validation: n >= 1, row_ptr[0] = 0,
 * non-decreasing, row_ptr[n] = nnz, col_idx < n, w >= 1; with
 * BC_UNDIRECTED_CHECK also the symmetry of the entries.  Precomputes
 * Delta_node(v) = min incident weight (Sec. 3.2, before Eq. 2).  Internal
 * vertex order is a layout choice only (see BC_RELABEL_DEGREE / BC_KEEP_ORDER):
 * every input and output of this ABI uses the caller's vertex and entry ids.
 * On success *out holds an opaque handle that bc_graph_destroy releases.
 */
int bc_graph_create(const uint64_t *row_ptr, const uint32_t *col_idx, const uint32_t *w, uint32_t n,
                    uint64_t nnz, uint32_t flags, bc_graph_t *out);

/* Release a graph.  Fails with BC_ERR_BUSY while serving requests still use it. */
int bc_graph_destroy(bc_graph_t g);

typedef struct bc_graph_info {
  uint32_t n;
  uint64_t nnz;
  uint32_t max_weight;
  uint32_t dist_bits;     /* 32 or 64: device distance width chosen for this graph */
  uint64_t device_bytes;  /* resident CSR + per-vertex graph data */
  uint64_t slab_bytes;    /* device bytes one in-flight source needs */
  uint32_t relabeled;     /* 1 when vertices are stored internally in decreasing-degree order */
  uint32_t directed;      /* 1 for a BC_DIRECTED graph */
} bc_graph_info;

int bc_graph_get_info(bc_graph_t g, bc_graph_info *out);

/*
 * Synchronous BC over a source list (Sec. 2.1, Algorithms 1-3).
 * sources[k] and out_bc[n] are HOST arrays owned by the caller; out_bc is
 * overwritten with scale * sum_s delta_s.  k = 0 yields all zeros.
 */
int bc_compute(bc_graph_t g, const uint32_t *sources, uint32_t k, double scale, double *out_bc);

/*
 * Asynchronous BC on a caller stream.  d_sources[k] and d_out_bc[n] are
 * DEVICE arrays owned by the caller (e.g. torch tensors); stream is a
 * cudaStream_t (NULL = legacy default stream).  Returns after enqueueing;
 * d_out_bc is valid once the stream reaches that point.  Sources are
 * validated on the device: an out-of-range source sets the graph's error word,
 * which bc_sync_status() reports as BC_ERR_INVALID.
 */
int bc_compute_async(bc_graph_t g, const uint32_t *d_sources, uint32_t k, double scale, double *d_out_bc,
                     void *stream);

/*
 * Wait for all work enqueued on `stream` by bc_compute_async for graph g and
 * return the status recorded by its kernels (BC_OK, BC_ERR_TIMEOUT, BC_ERR_INVALID).
 * Each stream that made an async call on g keeps one of g's workspaces (its
 * slabs and status block) reserved until this call, or the same stream's next
 * async call on g, has read that status: call bc_sync_status before
 * destroying the stream or reusing its handle, or the workspace stays reserved
 * (and the pool grows by one workspace for each such stream).  If the
 * synchronisation itself fails, the workspace is released and BC_ERR_CUDA
 * is returned.
 */
int bc_sync_status(bc_graph_t g, void *stream);

/*
 * Edge betweenness (the paper's tool reports node and edge BC, Sec. 1).
 * out_ebc[nnz] (HOST) receives, per CSR entry e = (a -> b, w):
 *   scale * sum_s sigma_sa / sigma_sb * (1 + delta_s(b))   when d(a) + w = d(b),
 * i.e. the dependency share that crosses the entry from a to b; 0 otherwise.
 * The undirected edge {a, b} carries the sum of its two entries.  out_bc[n]
 * (HOST, may be NULL) receives the vertex BC of the same run.
 */
int bc_edge_compute(bc_graph_t g, const uint32_t *sources, uint32_t k, double scale, double *out_ebc,
                    double *out_bc);

/* Edge BC with DEVICE buffers on the caller's stream (the bc_compute_async
 * form of bc_edge_compute): d_sources[k], d_out_ebc[nnz] (caller's entry ids)
 * and d_out_bc[n] are device arrays the caller owns; both outputs are
 * overwritten.  Status through bc_sync_status. */
int bc_edge_compute_async(bc_graph_t g, const uint32_t *d_sources, uint32_t k, double scale, double *d_out_ebc,
                          double *d_out_bc, void *stream);

/*
 * The paper's own thread mappings, for comparison (Sec. 3.1-3.4, Fig. 2-5):
 * one source at a time over the whole GPU; each phase expands the frontier
 * node-parallel (Algorithm 2: a group of vwarp threads per vertex of V,
 * node_parallel = 1) or work-efficient (Algorithms 4-5: groups only for the
 * frontier queue, node_parallel = 0) with vwarp in {1, 4, 8, 16, 32} threads
 * per vertex (1 = thread per vertex, otherwise the warp-centric mapping of
 * Sec. 3.4), then computes Delta_i (Eq. 2) and settles (Eq. 4) by scanning
 * all V.  Same results as bc_compute (exact distances, FP64 sigma and BC);
 * undirected graphs only.  sources[k] and out_bc[n] are HOST arrays.
 */
int bc_compute_paper_variant(bc_graph_t g, const uint32_t *sources, uint32_t k, double scale, double *out_bc,
                             int node_parallel, int vwarp);

/*
 * Serving (continuous batching).  Submit copies sources[k] at the call; the
 * HOST array out_bc[n] must stay valid until the request is DONE, FAILED or
 * CANCELLED.  Requests on different graphs and sizes are admitted in arrival
 * order as device memory allows (each holds a workspace for up to as many
 * sources in flight as the GPU holds for its graph).  Every admitted request
 * runs as a sequence of source batches (about two waves of its sources in
 * flight each); a scheduler thread interleaves the batches of all admitted
 * requests on up to 8 streams, earliest deadline first (submit time + the
 * request's entries to walk / the measured aggregate rate), and re-divides
 * the GPU's resident threads at every batch among the requests with work
 * left (at most 2 ways), so batches of different graphs run on the device at
 * the same time and a large request yields at its batch boundaries.  Not in
 * the paper: a serving layer around its per-source method.
 * BC_ERR_NOMEM: the request alone can never fit the memory budget.
 * BC_ERR_BUSY: the pending queue is full.
 */
int bc_request_submit(bc_graph_t g, const uint32_t *sources, uint32_t k, double scale, double *out_bc,
                      bc_request_t *out_id);

/* Current state of a request (BC_REQ_*); BC_ERR_INVALID for an unknown id. */
int bc_request_poll(bc_request_t id, int *out_state);

/*
 * Block until the request leaves QUEUED/RUNNING or timeout_ms passes
 * (timeout_ms < 0: no limit).  Returns BC_OK when DONE, the request's error
 * code when FAILED, BC_ERR_CANCELLED when cancelled, BC_ERR_TIMEOUT on timeout.
 * A request that has finished is forgotten after bc_request_wait returns.
 */
int bc_request_wait(bc_request_t id, int timeout_ms);

/* Cancel a request (BC_OK).  A QUEUED one is CANCELLED at once; a RUNNING one
 * stops at its next source-batch boundary and ends CANCELLED without writing
 * out_bc; a finished one is left as it is. */
int bc_request_cancel(bc_request_t id);

/* Serving statistics: requests completed and their latencies (submit -> done). */
typedef struct bc_serving_stats {
  uint64_t completed;
  uint64_t failed;
  double p50_ms;
  double p99_ms;
  double mean_ms;
  uint64_t edges_traversed; /* sum over completed requests of k * (nnz / 2) */
  uint32_t max_concurrent;  /* largest number of requests seen running at once */
} bc_serving_stats;

int bc_serving_stats_get(bc_serving_stats *out);
int bc_serving_reset(void);

/*
 * Test hook: distances (UINT64_MAX = unreachable), shortest-path counts and
 * the settle batch (level) of every vertex from one source, as the batched
 * path computes them (Algorithm 2 semantics, strict criterion).  HOST outputs
 * of n entries each; any may be NULL.  Unreached vertices get level
 * UINT32_MAX.  Within a source, every shortest-path DAG edge (p -> v)
 * satisfies level[p] < level[v].
 */
int bc_sssp_debug(bc_graph_t g, uint32_t s, uint64_t *out_dist, double *out_sigma, uint32_t *out_level);

/*
 * Per-run counters of the last batched run on this thread's last-used graph:
 * phases (settle batches) summed over sources, near/far refills, levels,
 * relaxations attempted (atomicMin issued) and reached vertices.
 */
typedef struct bc_run_stats {
  uint64_t sources;
  uint64_t phases;
  uint64_t refills;
  uint64_t reached;
  uint64_t relax_atomics;
  uint64_t entries_scanned;
  uint32_t team_threads;
  uint32_t slots;
  uint64_t bucket_width;
  uint64_t dag_edges;       /* shortest-path DAG edges recorded by the forward pass */
  uint64_t pair_overflows;  /* sources whose DAG edge list overflowed (backward fell back to a CSR scan) */
  uint64_t cycles_expand;   /* SM cycles summed over sources: frontier expansion (sigma pull + relax) */
  uint64_t cycles_refill;   /* near-queue refills from the far queue */
  uint64_t cycles_settle;   /* threshold + settle of the near queue */
  uint64_t cycles_backward; /* dependency accumulation */
  uint64_t near_scanned;    /* near-queue entries read by threshold and settle */
  uint64_t far_scanned;     /* far-queue entries read by refills */
  uint64_t levels;          /* backward levels summed over sources (settle batches, or DAG hop depths) */
  uint32_t algorithm;       /* schedule of the run: BC_ALGO_STRICT or BC_ALGO_DELTA */
  uint32_t warp_degree;     /* degree thresholds of the run's forward expansion: rows with at least */
  uint32_t team_degree;     /* warp_degree entries got a warp each, with at least team_degree the whole team */
  uint32_t settle_in;       /* settle test of the run (bc_config.settle_in values 1, 2 or 3) */
} bc_run_stats;

int bc_last_run_stats(bc_graph_t g, bc_run_stats *out);

/*
 * Autotuner: times candidate settings on a probe sample of `sources`
 * (k_probe of them, HOST array) and stores the fastest as the graph's tuned
 * configuration, used whenever the process-wide config leaves a field at 0:
 * team size x bucket width (and the delta-stepping schedule where the strict
 * one needs 1000 or more phases per source), then the degree thresholds of
 * the forward expansion (warp_degree in {8, 16, 32, 64}, then team_degree in
 * {2, 8, 32} x team size; Sec. 3.4 studies the same trade-off as its
 * WARP_SIZE), then sources in flight (full or half capacity).  Results are
 * cached per graph fingerprint.
 */
int bc_autotune(bc_graph_t g, const uint32_t *sources, uint32_t k_probe);

/*
 * Step graphs: one batched run (Algorithms 1-3 for every source of a fixed
 * list, Sec. 3.1's block-per-source batching) captured once as a CUDA graph
 * and replayed with a single launch.  The step is bound to DEVICE buffers
 * that the caller owns and keeps alive until bc_step_destroy: d_sources[k]
 * (read at every launch, so the caller may rewrite the ids in place between
 * launches) and d_out_bc[n] (zeroed, accumulated and scaled at every launch,
 * caller's vertex ids).  The configuration (team size, width, schedule, slots)
 * is the one in effect at creation.  The step owns its workspace: launches of
 * one step must be ordered (one stream, or caller-ordered streams); different
 * steps run concurrently.  bc_step_launch returns once the graph is enqueued
 * on `stream` (a cudaStream_t, NULL = legacy default); bc_step_sync waits for
 * the stream and returns the device status of the last launch (BC_ERR_INVALID
 * for a source >= n, BC_ERR_TIMEOUT for a phase cap hit; the step stays usable)
 * and records bc_last_run_stats.  bc_graph_destroy fails with BC_ERR_BUSY
 * while steps of the graph exist.
 */
typedef struct bc_step *bc_step_t;
int bc_step_create(bc_graph_t g, const uint32_t *d_sources, uint32_t k, double scale, double *d_out_bc,
                   bc_step_t *out);
int bc_step_launch(bc_step_t step, void *stream);
int bc_step_sync(bc_step_t step, void *stream);
int bc_step_destroy(bc_step_t step);

/*
 * No-allocation variant of bc_compute_async, for callers that cannot allocate
 * device memory while they run (a host thread with real-time limits, code
 * running while another framework owns the device allocator, a process whose
 * memory is reserved up front).  The paper has no counterpart: it is an
 * interface addition.
 *
 * Inputs and outputs are the caller's DEVICE arrays: the CSR of the
 * undirected graph (d_row_ptr[n + 1], d_col_idx[nnz], d_w[nnz], the same
 * conventions as bc_graph_create, both directions of every edge stored; the
 * contents are validated on the device: row_ptr, col_idx < n, w >= 1, every
 * source < n, and symmetry, by comparing a 64-bit hash sum of all entries
 * with that of their reverses, so a CSR with a one-way entry is reported as
 * BC_ERR_INVALID except with probability about 2^-64),
 * d_sources[k], d_out_bc[n] (overwritten with scale * sum_s delta_s, in the
 * caller's vertex ids) and d_status (one int, set to BC_OK, BC_ERR_INVALID or
 * BC_ERR_TIMEOUT when the work completes).  Work is enqueued on `stream`
 * (a cudaStream_t) and the call returns without waiting.
 *
 * All scratch lives in one fixed device array of BC_NOALLOC_SCRATCH_BYTES
 * that every GPU loading this library holds until the process exits; the call
 * makes no cudaMalloc or cudaFree and calls no allocating routine.  A graph
 * whose packed CSR, per-vertex data and one per-source slab do not fit is
 * rejected with BC_ERR_NOMEM before any device work; fewer sources then run
 * at once when only a few slabs fit.  Distances use 64-bit words.
 *
 * The first call on a device looks up the array's device address, so make it
 * before any stream capture.  Calls share the array and each re-initialises
 * it; calls whose work overlaps on the GPU (other streams or threads without
 * ordering) race on it.  On BC_ERR_INVALID no source runs and d_out_bc is all
 * zeros.  The bc_config fields that apply: bucket_width (0 = a fixed 64: the
 * call never reads the weights on the host, so it cannot derive the mean
 * Delta_node that bc_compute uses; pass the graph's own width for high-weight
 * graphs), settle_in, phase_cap, warp_degree and team_degree.  The team size
 * follows the average degree (>= 20: 512, >= 12: 256, else 128 threads); the
 * other fields are ignored.
 */
#define BC_NOALLOC_SCRATCH_BYTES (64ull << 20)
int bc_compute_noalloc(const uint64_t *d_row_ptr, const uint32_t *d_col_idx, const uint32_t *d_w, uint32_t n,
                       uint64_t nnz, const uint32_t *d_sources, uint32_t k, double scale, double *d_out_bc,
                       int *d_status, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BCGPU_H */
