// bc_compute_noalloc: batched BC with no device allocation at call time.
//
// Who needs it: callers that must not allocate device memory while they run,
// for example a host thread with real-time limits, code that runs while
// another framework owns the device allocator, or a process whose memory is
// fully reserved up front.  Such callers cannot create a bc_graph_t (that
// allocates), so this entry point takes the caller's device CSR directly.
//
// All scratch (the packed adjacency, Delta_node, the control block and the
// per-source slabs) lives in one file-scope device array of
// BC_NOALLOC_SCRATCH_BYTES.  Every GPU that loads the library holds this
// array until the process exits.  The host code never uses the symbol itself
// as an address: once per device, with that device current, it asks the
// runtime for the array's device address (cudaGetSymbolAddress) and passes that
// pointer to the kernels.  The first call on a device does this set-up, so it
// should come before any stream capture.  The address is cached per device
// together with the unique id of the context it was looked up in; a call
// that finds another context current (for example after cudaDeviceReset)
// looks the address up again.
//
// All calls share the array, and it keeps whatever the last call left there.
// Each call therefore re-initialises what must start at a known value: the
// control block, the distance words (INF) and the backward accumulators (0).
// Two calls whose work overlaps on the GPU (different streams, or different
// host threads, without ordering between them) race on the array.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/bcgpu.h"
#include "bc_common.h"

namespace bcgpu {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[BC_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_na_mu;

// The scratch array's device address on each device, and the unique id of the
// context it was looked up in (0: unknown, look it up again).
struct NaAddr {
  unsigned long long ctx_id;
  char* ptr;
};
NaAddr g_na_addr[kMaxDevices] = {};

// cuCtxGetCurrent and cuCtxGetId, reached through the runtime's driver entry
// point query so the library needs no link-time dependency on the driver.
using CtxGetCurrentFn = int (*)(void** ctx);
using CtxGetIdFn = int (*)(void* ctx, unsigned long long* id);

// Unique id of the calling thread's current context, or 0 when none is
// current yet or the driver does not offer the query.
unsigned long long current_ctx_id() {
  static const CtxGetCurrentFn get_cur = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<CtxGetCurrentFn>(f);
  }();
  static const CtxGetIdFn get_id = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<CtxGetIdFn>(f);
  }();
  if (!get_cur || !get_id) return 0;
  void* ctx = nullptr;
  if (get_cur(&ctx) != 0 || !ctx) return 0;
  unsigned long long id = 0;
  if (get_id(ctx, &id) != 0) return 0;
  return id;
}

struct NaCtl {
  uint32_t counter;
  int err;
  uint32_t debug[2];
  unsigned long long stats[STAT_COUNT];
  // sums over all entries (v -> u, w) of hash(v, u, w) and of hash(u, v, w):
  // equal for a symmetric CSR (the two multisets are the same)
  unsigned long long sym[2];
};

// The device status word carries DEV_* codes; the caller reads them as BC_* codes.
static_assert(DEV_OK == BC_OK && DEV_ERR_INVALID == BC_ERR_INVALID && DEV_ERR_TIMEOUT == BC_ERR_TIMEOUT,
              "device status codes must equal the ABI codes they are reported as");

constexpr uint64_t kCtlBytes = 256;
static_assert(sizeof(NaCtl) <= kCtlBytes, "control block must fit its reserved bytes");

uint64_t al256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

// Per-source slab with 64-bit distances (weights are not inspected on the
// host, so the wide distance type is always safe).
SlabLayout na_layout(uint32_t n) {
  SlabLayout L{};
  uint64_t off = 0;
  L.off_d = off;
  off += al256((uint64_t)n * 8);
  L.off_sig = off;
  off += al256((uint64_t)n * 8);
  L.off_S = off;
  off += al256((uint64_t)n * 4);
  L.off_ends = off;
  off += al256(((uint64_t)n + 2) * 4);
  L.off_near = off;
  off += al256((uint64_t)n * 4);
  L.off_far = off;
  off += al256((uint64_t)n * 4);
  L.off_far2 = off;
  off += al256((uint64_t)n * 4);
  L.off_acc = off;
  off += al256((uint64_t)n * 8);
  L.off_pend = off;
  off += al256(((uint64_t)n + 2) * 4);
  L.pair_cap = (uint32_t)std::min<uint64_t>(2ull * n + 64, 0xffffffffull);
  L.off_pairs = off;
  off += al256((uint64_t)L.pair_cap * 8);
  L.off_pc = off;
  off += al256((uint64_t)n * 4);
  L.stride = off;
  return L;
}

// 64-bit finaliser of SplitMix64 (Steele, Lea and Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Hash of one directed entry (a -> b, weight w).
__device__ __forceinline__ uint64_t entry_hash(uint32_t a, uint32_t b, uint32_t w) {
  return mix64((((uint64_t)a << 32) | b) ^ mix64((uint64_t)w + 0x9e3779b97f4a7c15ull));
}

// Validates the caller's CSR while packing it (every read stays inside the
// caller's arrays whatever their contents) and computes Delta_node.  On any
// violation it records DEV_ERR_INVALID and parks the source counter far above
// any source index, so the batched kernel that follows does no work.  It also
// sums, mod 2^64, a hash of every entry (v -> u, w) and of its reverse
// (u -> v, w); na_check_symmetry compares the two sums.
__global__ void na_validate_prep(uint32_t n, uint64_t nnz, const uint64_t* __restrict__ row_ptr,
                                 const uint32_t* __restrict__ col, const uint32_t* __restrict__ w,
                                 const uint32_t* __restrict__ src, uint32_t k, uint2* __restrict__ adj,
                                 uint32_t* __restrict__ dnode, NaCtl* ctl) {
  const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
  bool bad = false;
  unsigned long long fwd = 0, rev = 0;
  if (tid == 0 && (row_ptr[0] != 0 || row_ptr[n] != nnz)) bad = true;
  for (uint64_t v = tid; v < n; v += nth) {
    const uint64_t r0 = row_ptr[v], r1 = row_ptr[v + 1];
    uint32_t m = 0xffffffffu;
    if (r0 > r1 || r1 > nnz) {
      bad = true;
    } else {
      for (uint64_t e = r0; e < r1; ++e) {
        const uint32_t c = col[e], ww = w[e];
        if (c >= n || ww == 0) bad = true;
        adj[e] = make_uint2(c < n ? c : 0u, ww);
        m = min(m, ww);
        fwd += entry_hash((uint32_t)v, c, ww);
        rev += entry_hash(c, (uint32_t)v, ww);
      }
    }
    dnode[v] = m;
  }
  for (uint64_t i = tid; i < k; i += nth)
    if (src[i] >= n) bad = true;
  for (int o = 16; o > 0; o >>= 1) {
    fwd += __shfl_xor_sync(0xffffffffu, fwd, o);
    rev += __shfl_xor_sync(0xffffffffu, rev, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&ctl->sym[0], fwd);
    atomicAdd(&ctl->sym[1], rev);
  }
  if (bad) {
    atomicCAS(&ctl->err, DEV_OK, DEV_ERR_INVALID);
    atomicExch(&ctl->counter, 0x80000000u);
  }
}

// An asymmetric CSR (some entry without its reverse entry of the same
// weight) makes the two hash sums differ; it is then rejected like any other
// invalid input.  Single thread.
__global__ void na_check_symmetry(NaCtl* ctl) {
  if (ctl->sym[0] != ctl->sym[1]) {
    atomicCAS(&ctl->err, DEV_OK, DEV_ERR_INVALID);
    atomicExch(&ctl->counter, 0x80000000u);
  }
}

int na_fail(int code, const char* msg) { return set_error(code, msg); }

}  // namespace
}  // namespace bcgpu

using namespace bcgpu;

extern "C" int bc_compute_noalloc(const uint64_t* d_row_ptr, const uint32_t* d_col_idx, const uint32_t* d_w,
                                  uint32_t n, uint64_t nnz, const uint32_t* d_sources, uint32_t k, double scale,
                                  double* d_out_bc, int* d_status, void* stream) {
  if (n == 0 || n > 0xfffffff0u) return na_fail(BC_ERR_INVALID, "bc_compute_noalloc: n must be in [1, 2^32 - 16]");
  if (!d_row_ptr || !d_out_bc || !d_status) return na_fail(BC_ERR_INVALID, "bc_compute_noalloc: null pointer");
  if (nnz > 0 && (!d_col_idx || !d_w)) return na_fail(BC_ERR_INVALID, "bc_compute_noalloc: null col_idx or w");
  if (k > 0 && !d_sources) return na_fail(BC_ERR_INVALID, "bc_compute_noalloc: null sources");
  if (nnz >= (1ull << 32)) return na_fail(BC_ERR_INVALID, "bc_compute_noalloc: nnz must be below 2^32");
  if (k >= 0x80000000u) return na_fail(BC_ERR_INVALID, "bc_compute_noalloc: k must be below 2^31");
  const SlabLayout lay = na_layout(n);
  const uint64_t off_adj = kCtlBytes;
  const uint64_t off_dnode = off_adj + al256(std::max<uint64_t>(nnz, 1) * 8);
  const uint64_t off_slabs = off_dnode + al256((uint64_t)n * 4);
  if (off_slabs + lay.stride > BC_NOALLOC_SCRATCH_BYTES) {
    char msg[256];
    snprintf(msg, sizeof msg,
             "bc_compute_noalloc: graph needs %llu scratch bytes for one source, above the fixed maximum of %llu "
             "(BC_NOALLOC_SCRATCH_BYTES); use bc_graph_create + bc_compute_async",
             (unsigned long long)(off_slabs + lay.stride), (unsigned long long)BC_NOALLOC_SCRATCH_BYTES);
    return na_fail(BC_ERR_NOMEM, msg);
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(BC_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return na_fail(BC_ERR_INVALID, "bc_compute_noalloc: device index too large");
  char* base = nullptr;
  {
    // set-up, once per device and context: the array's device address
    std::lock_guard<std::mutex> lk(g_na_mu);
    NaAddr& ad = g_na_addr[dev];
    const unsigned long long cur = current_ctx_id();
    if (!ad.ptr || cur == 0 || cur != ad.ctx_id) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // makes the device's context current if needed
      if (e != cudaSuccess) return na_fail(BC_ERR_CUDA, cudaGetErrorString(e));
      ad.ptr = static_cast<char*>(p);
      ad.ctx_id = current_ctx_id();
    }
    base = ad.ptr;
  }
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return na_fail(BC_ERR_CUDA, cudaGetErrorString(e));
  const double avg_deg = (double)nnz / n;
  const int team = avg_deg >= 20.0 ? 512 : (avg_deg >= 12.0 ? 256 : 128);
  int bps = 0;
  e = batched_occupancy(64, team, &bps);
  if (e != cudaSuccess) return na_fail(BC_ERR_CUDA, cudaGetErrorString(e));
  const uint32_t per_block = (uint32_t)(batched_block_threads(team) / team);
  uint64_t slots = (uint64_t)std::max(bps, 1) * sms * per_block;
  slots = std::min<uint64_t>(slots, (BC_NOALLOC_SCRATCH_BYTES - off_slabs) / lay.stride);
  slots = std::min<uint64_t>(slots, std::max<uint32_t>(k, 1));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  NaCtl* ctl = reinterpret_cast<NaCtl*>(base);
  uint2* adj = reinterpret_cast<uint2*>(base + off_adj);
  uint32_t* dnode = reinterpret_cast<uint32_t*>(base + off_dnode);
  char* slabs = base + off_slabs;
  bc_config cfg;
  bc_get_config(&cfg);

  e = cudaMemsetAsync(ctl, 0, sizeof(NaCtl), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_out_bc, 0, (size_t)n * 8, st);
  if (e == cudaSuccess) {
    const uint64_t work = std::max<uint64_t>(n, k);
    const int grid = (int)std::min<uint64_t>((work + 255) / 256, (uint64_t)sms * 8);
    na_validate_prep<<<std::max(grid, 1), 256, 0, st>>>(n, nnz, d_row_ptr, d_col_idx, d_w, d_sources, k, adj, dnode,
                                                        ctl);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    na_check_symmetry<<<1, 1, 0, st>>>(ctl);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = launch_fill_slabs(slabs, lay.stride, (uint32_t)slots, lay.off_d, al256((uint64_t)n * 8),
                                              0xffffffffu, st);
  if (e == cudaSuccess)
    e = launch_fill_slabs(slabs, lay.stride, (uint32_t)slots, lay.off_acc, al256((uint64_t)n * 8), 0u, st);
  if (e == cudaSuccess)
    e = launch_fill_slabs(slabs, lay.stride, (uint32_t)slots, lay.off_pc, al256((uint64_t)n * 4), 0u, st);
  if (e == cudaSuccess) {
    BatchArgs a{};
    a.g.n = n;
    a.g.nnz = nnz;
    a.g.row_ptr = d_row_ptr;
    a.g.adj = adj;
    a.g.adjp = nullptr;
    a.g.dnode = dnode;
    a.sources = d_sources;
    a.k = k;
    a.counter = &ctl->counter;
    a.bc = d_out_bc;
    a.ebc = nullptr;
    a.slabs = slabs;
    a.lay = lay;
    a.nslots = (uint32_t)slots;
    a.width = cfg.bucket_width ? cfg.bucket_width : 64;
    a.settle_in = cfg.settle_in == 2 ? 0u : 1u;
    a.phase_cap = cfg.phase_cap ? cfg.phase_cap : 4ull * n + 64;  // phases + refills <= 4n + 2
    a.err = &ctl->err;
    a.stats = ctl->stats;
    a.flags = 0;
    a.debug_out = ctl->debug;
    a.algo = ALGO_STRICT;
    a.warp_deg = cfg.warp_degree ? cfg.warp_degree : 32u;
    a.team_deg = std::max<uint32_t>(cfg.team_degree ? cfg.team_degree : 8u * team, a.warp_deg);
    const int grid = (int)((slots + per_block - 1) / per_block);
    e = launch_batched(a, 64, team, grid, st);
  }
  if (e == cudaSuccess && scale != 1.0) e = launch_scale(d_out_bc, n, scale, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_status, &ctl->err, sizeof(int), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return na_fail(BC_ERR_CUDA, cudaGetErrorString(e));
  return BC_OK;
}
