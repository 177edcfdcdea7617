// Plain form: one source at a time, every phase a set of whole-GPU kernel
// launches driven from the host (the straightforward mapping of Algorithms
// 2 and 3 of arxiv 1701.05975, with the work-efficient frontier queue of
// Algorithms 4-5 and a warp per frontier vertex, the warp-centric expansion
// of Sec. 3.4).  Same settle rule, near/far queues, sigma pull and backward
// pull as the batched kernel; it exists as the baseline the batched form is
// measured against.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>
#include <vector>

#include "bc_common.h"

namespace bcgpu {

struct PlainCtr {
  unsigned long long out_min, dmin, fmin, split;
  unsigned int near_len, far_len, near_out, far_out, S_len, pad;
};

struct PlainWork {
  uint32_t n;
  int dist_bits;
  void* d;
  double* sig;
  uint32_t* S;
  uint32_t* nearq[2];
  uint32_t* farq[2];
  PlainCtr* ctr;
  PlainCtr* host_ctr;  // pinned
};

namespace {

constexpr unsigned FULL = 0xffffffffu;

template <typename D>
__device__ __forceinline__ D dinf() {
  return ~D(0);
}
__device__ __forceinline__ uint32_t ldcg(const uint32_t* p) { return __ldcg(p); }
__device__ __forceinline__ uint64_t ldcg(const uint64_t* p) {
  return (uint64_t)__ldcg(reinterpret_cast<const unsigned long long*>(p));
}
__device__ __forceinline__ uint32_t amin(uint32_t* p, uint32_t v) { return atomicMin(p, v); }
__device__ __forceinline__ uint64_t amin(uint64_t* p, uint64_t v) {
  return (uint64_t)atomicMin(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}
template <typename D>
__device__ __forceinline__ D sat_add(uint64_t a, uint64_t b) {
  const uint64_t lim = (uint64_t)dinf<D>() - 1;
  if (a >= lim || b >= lim - a) return (D)lim;
  return (D)(a + b);
}

template <typename D>
__global__ void init_kernel(D* d, double* sig, uint32_t* S, PlainCtr* c, uint32_t s, uint64_t width) {
  d[s] = 0;
  sig[s] = 1.0;
  S[0] = s;
  c->near_len = c->far_len = c->near_out = c->far_out = 0;
  c->S_len = 1;
  c->split = sat_add<D>(0, width);
}

// ops on the control block between phases
enum { CTL_PRE_THRESHOLD = 0, CTL_POST_SETTLE, CTL_PRE_REFILL, CTL_POST_REFILL };

template <typename D>
__global__ void ctl_kernel(PlainCtr* c, int op, uint64_t width) {
  switch (op) {
    case CTL_PRE_THRESHOLD:
      c->out_min = c->dmin = ~0ull;
      c->near_out = 0;
      break;
    case CTL_POST_SETTLE:
      c->near_len = c->near_out;
      break;
    case CTL_PRE_REFILL:
      c->fmin = ~0ull;
      c->far_out = 0;
      break;
    case CTL_POST_REFILL:
      c->far_len = c->far_out;
      if (c->fmin != ~0ull) c->split = sat_add<D>(c->fmin, width);
      break;
  }
}

// One warp per frontier vertex: sigma pull from predecessors, relax the rest.
template <typename D>
__global__ void expand_kernel(GraphDev g, D* d, double* sig, const uint32_t* S, uint32_t f0, uint32_t f1, uint32_t s,
                              uint32_t* nearq, uint32_t* farq, PlainCtr* c) {
  const D INF = dinf<D>();
  const D split = (D)c->split;
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t i = f0 + warp; i < f1; i += nwarps) {
    const uint32_t v = S[i];
    const D dv = ldcg(&d[v]);
    double acc = 0.0;
    for (uint64_t e = g.row_ptr[v] + lane; e < g.row_ptr[v + 1]; e += 32) {
      const uint2 ent = g.adjp ? make_uint2(g.adjp[e] & ((1u << g.col_bits) - 1u), g.adjp[e] >> g.col_bits)
                                     : g.adj[e];
      const uint32_t u = ent.x;
      const D w = (D)ent.y;
      const D du = ldcg(&d[u]);
      if (du != INF && du + w == dv) {
        acc += __ldcg(&sig[u]);
      } else {
        const D nd = dv + w;
        if (nd < du) {
          const D old = amin(&d[u], nd);
          if (nd < old) {
            if (old == INF) {
              if (nd < split) nearq[atomicAdd(&c->near_len, 1u)] = u;
              else farq[atomicAdd(&c->far_len, 1u)] = u;
            } else if (old >= split && nd < split) {
              nearq[atomicAdd(&c->near_len, 1u)] = u;
            }
          }
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if (lane == 0 && v != s) sig[v] = acc;
  }
}

template <typename D>
__global__ void far_min_kernel(const D* d, const uint32_t* farq, PlainCtr* c) {
  const D old = (D)c->split;
  const uint32_t fl = c->far_len;
  unsigned long long m = ~0ull;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < fl; j += gridDim.x * blockDim.x) {
    const D du = ldcg(&d[farq[j]]);
    if (du >= old && (unsigned long long)du < m) m = du;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(FULL, m, o));
  if ((threadIdx.x & 31) == 0 && m != ~0ull) atomicMin(&c->fmin, m);
}

template <typename D>
__global__ void far_partition_kernel(const D* d, const uint32_t* farq, uint32_t* nearq, uint32_t* farq_out,
                                     PlainCtr* c, uint64_t width) {
  const D old = (D)c->split;
  const D ns = c->fmin == ~0ull ? old : sat_add<D>(c->fmin, width);
  const uint32_t fl = c->far_len;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < fl; j += gridDim.x * blockDim.x) {
    const uint32_t u = farq[j];
    const D du = ldcg(&d[u]);
    if (du < old) continue;
    if (du < ns) nearq[atomicAdd(&c->near_len, 1u)] = u;
    else farq_out[atomicAdd(&c->far_out, 1u)] = u;
  }
}

template <typename D>
__global__ void threshold_kernel(const D* d, const uint32_t* dnode, const uint32_t* nearq, PlainCtr* c) {
  const uint32_t nl = c->near_len;
  unsigned long long o = ~0ull, m = ~0ull;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < nl; j += gridDim.x * blockDim.x) {
    const uint32_t u = nearq[j];
    const D du = ldcg(&d[u]);
    o = min(o, (unsigned long long)(du + (D)dnode[u]));
    m = min(m, (unsigned long long)du);
  }
#pragma unroll
  for (int k = 16; k > 0; k >>= 1) {
    o = min(o, __shfl_xor_sync(FULL, o, k));
    m = min(m, __shfl_xor_sync(FULL, m, k));
  }
  if ((threadIdx.x & 31) == 0) {
    if (o != ~0ull) atomicMin(&c->out_min, o);
    if (m != ~0ull) atomicMin(&c->dmin, m);
  }
}

template <typename D>
__global__ void settle_kernel(const D* d, const uint32_t* dnode, const uint32_t* nearq, uint32_t* nearq_out,
                              uint32_t* S, PlainCtr* c, uint32_t settle_in) {
  const uint32_t nl = c->near_len;
  const unsigned long long thr = min(c->out_min, c->split);
  const unsigned long long dm = c->dmin;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < nl; j += gridDim.x * blockDim.x) {
    const uint32_t u = nearq[j];
    const unsigned long long du = ldcg(&d[u]);
    bool take = du < thr;
    if (settle_in && !take) take = du < dm + dnode[u];
    if (take) S[atomicAdd(&c->S_len, 1u)] = u;
    else nearq_out[atomicAdd(&c->near_out, 1u)] = u;
  }
}

// Algorithm 3 for one level, one warp per vertex.
template <typename D>
__global__ void backward_kernel(GraphDev g, const D* d, double* sig, const uint32_t* S, uint32_t b0, uint32_t b1,
                                double* bc) {
  const D INF = dinf<D>();
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t i = b0 + warp; i < b1; i += nwarps) {
    const uint32_t v = S[i];
    const D dv = d[v];
    double acc = 0.0;
    for (uint64_t e = g.row_ptr[v] + lane; e < g.row_ptr[v + 1]; e += 32) {
      const uint2 ent = g.adjp ? make_uint2(g.adjp[e] & ((1u << g.col_bits) - 1u), g.adjp[e] >> g.col_bits)
                                     : g.adj[e];
      const D du = d[ent.x];
      if (du != INF && du == dv + (D)ent.y) acc += sig[ent.x];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if (lane == 0) {
      const double sg = sig[v];
      const double delta = sg * acc;
      sig[v] = (1.0 + delta) / sg;
      atomicAdd(&bc[g.n2o ? g.n2o[v] : v], delta);
    }
  }
}

template <typename D>
__global__ void reset_kernel(D* d, const uint32_t* S, uint32_t len) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < len; j += gridDim.x * blockDim.x) d[S[j]] = dinf<D>();
}

template <typename D>
__global__ void fill_kernel(D* d, uint32_t n) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) d[j] = dinf<D>();
}

inline int blocks_for(uint64_t items, int per_block, int cap) {
  uint64_t b = (items + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > (uint64_t)cap) b = cap;
  return (int)b;
}

#define PCHK(x)                     \
  do {                              \
    cudaError_t e_ = (x);           \
    if (e_ != cudaSuccess) return e_; \
  } while (0)

template <typename D>
cudaError_t run_t(PlainWork* w, const GraphDev& g, const uint32_t* src, const uint32_t* host_o2n, uint32_t k,
                  double* bc, uint64_t width, uint32_t settle_in, uint64_t phase_cap, int sm_count, cudaStream_t st,
                  int* dev_status, unsigned long long* stats) {
  D* d = static_cast<D*>(w->d);
  const int cap = sm_count * 8;
  *dev_status = DEV_OK;
  for (uint32_t i = 0; i < k; ++i) {
    if (src[i] >= g.n) {
      *dev_status = DEV_ERR_INVALID;
      return cudaSuccess;
    }
    const uint32_t s = host_o2n ? host_o2n[src[i]] : src[i];
    int cn = 0, cf = 0;  // current near / far buffers
    init_kernel<D><<<1, 1, 0, st>>>(d, w->sig, w->S, w->ctr, s, width);
    PCHK(cudaGetLastError());
    std::vector<uint32_t> ends = {0, 1};
    uint32_t f0 = 0, f1 = 1;
    uint64_t phases = 0, refills = 0;
    bool timeout = false;
    for (;;) {
      expand_kernel<D><<<blocks_for((uint64_t)(f1 - f0) * 32, 256, cap), 256, 0, st>>>(
          g, d, w->sig, w->S, f0, f1, s, w->nearq[cn], w->farq[cf], w->ctr);
      PCHK(cudaGetLastError());
      PCHK(cudaMemcpyAsync(w->host_ctr, w->ctr, sizeof(PlainCtr), cudaMemcpyDeviceToHost, st));
      PCHK(cudaStreamSynchronize(st));
      while (w->host_ctr->near_len == 0 && w->host_ctr->far_len > 0) {
        const uint32_t fl = w->host_ctr->far_len;
        ctl_kernel<D><<<1, 1, 0, st>>>(w->ctr, CTL_PRE_REFILL, width);
        far_min_kernel<D><<<blocks_for(fl, 256, cap), 256, 0, st>>>(d, w->farq[cf], w->ctr);
        far_partition_kernel<D><<<blocks_for(fl, 256, cap), 256, 0, st>>>(d, w->farq[cf], w->nearq[cn],
                                                                           w->farq[cf ^ 1], w->ctr, width);
        ctl_kernel<D><<<1, 1, 0, st>>>(w->ctr, CTL_POST_REFILL, width);
        PCHK(cudaGetLastError());
        cf ^= 1;
        PCHK(cudaMemcpyAsync(w->host_ctr, w->ctr, sizeof(PlainCtr), cudaMemcpyDeviceToHost, st));
        PCHK(cudaStreamSynchronize(st));
        if (++refills + phases > phase_cap) {
          timeout = true;
          break;
        }
      }
      if (timeout || w->host_ctr->near_len == 0) break;
      const uint32_t nl = w->host_ctr->near_len;
      ctl_kernel<D><<<1, 1, 0, st>>>(w->ctr, CTL_PRE_THRESHOLD, width);
      threshold_kernel<D><<<blocks_for(nl, 256, cap), 256, 0, st>>>(d, g.dnode, w->nearq[cn], w->ctr);
      settle_kernel<D><<<blocks_for(nl, 256, cap), 256, 0, st>>>(d, g.dnode, w->nearq[cn], w->nearq[cn ^ 1], w->S,
                                                                 w->ctr, settle_in);
      ctl_kernel<D><<<1, 1, 0, st>>>(w->ctr, CTL_POST_SETTLE, width);
      PCHK(cudaGetLastError());
      cn ^= 1;
      PCHK(cudaMemcpyAsync(w->host_ctr, w->ctr, sizeof(PlainCtr), cudaMemcpyDeviceToHost, st));
      PCHK(cudaStreamSynchronize(st));
      ++phases;
      f0 = f1;
      f1 = w->host_ctr->S_len;
      ends.push_back(f1);
      if (phases + refills > phase_cap) {
        timeout = true;
        break;
      }
    }
    if (timeout) {
      fill_kernel<D><<<blocks_for(w->n, 256, cap), 256, 0, st>>>(d, w->n);
      PCHK(cudaGetLastError());
      PCHK(cudaStreamSynchronize(st));
      *dev_status = DEV_ERR_TIMEOUT;
      return cudaSuccess;
    }
    for (size_t lev = ends.size() - 2; lev >= 1; --lev) {
      const uint32_t b0 = ends[lev], b1 = ends[lev + 1];
      backward_kernel<D><<<blocks_for((uint64_t)(b1 - b0) * 32, 256, cap), 256, 0, st>>>(g, d, w->sig, w->S, b0, b1,
                                                                                           bc);
    }
    PCHK(cudaGetLastError());
    const uint32_t reached = ends.back();
    reset_kernel<D><<<blocks_for(reached, 256, cap), 256, 0, st>>>(d, w->S, reached);
    PCHK(cudaGetLastError());
    if (stats) {
      stats[STAT_SOURCES] += 1;
      stats[STAT_PHASES] += phases;
      stats[STAT_REFILLS] += refills;
      stats[STAT_REACHED] += reached;
    }
  }
  return cudaStreamSynchronize(st);
}

}  // namespace

uint64_t plain_bytes(uint32_t n, int dist_bits) {
  return (uint64_t)n * ((dist_bits / 8) + 8 + 4 + 4 * 4) + sizeof(PlainCtr) + 4096;
}

PlainWork* plain_create(uint32_t n, int dist_bits, cudaError_t* e) {
  PlainWork* w = new PlainWork();
  w->n = n;
  w->dist_bits = dist_bits;
  *e = cudaMalloc(&w->d, (size_t)n * (dist_bits / 8));
  if (*e == cudaSuccess) *e = cudaMalloc(&w->sig, (size_t)n * 8);
  if (*e == cudaSuccess) *e = cudaMalloc(&w->S, (size_t)n * 4);
  for (int i = 0; i < 2 && *e == cudaSuccess; ++i) {
    *e = cudaMalloc(&w->nearq[i], (size_t)n * 4);
    if (*e == cudaSuccess) *e = cudaMalloc(&w->farq[i], (size_t)n * 4);
  }
  if (*e == cudaSuccess) *e = cudaMalloc(&w->ctr, sizeof(PlainCtr));
  if (*e == cudaSuccess) *e = cudaMallocHost(&w->host_ctr, sizeof(PlainCtr));
  if (*e == cudaSuccess) *e = cudaMemset(w->d, 0xff, (size_t)n * (dist_bits / 8));
  if (*e == cudaSuccess) *e = cudaDeviceSynchronize();
  if (*e != cudaSuccess) {
    plain_destroy(w);
    return nullptr;
  }
  return w;
}

void plain_destroy(PlainWork* w) {
  if (!w) return;
  cudaFree(w->d);
  cudaFree(w->sig);
  cudaFree(w->S);
  for (int i = 0; i < 2; ++i) {
    cudaFree(w->nearq[i]);
    cudaFree(w->farq[i]);
  }
  cudaFree(w->ctr);
  if (w->host_ctr) cudaFreeHost(w->host_ctr);
  delete w;
}

cudaError_t plain_run(PlainWork* w, const GraphDev& g, int dist_bits, const uint32_t* host_sources,
                      const uint32_t* host_o2n, uint32_t k, double* bc, uint64_t width, uint32_t settle_in,
                      uint64_t phase_cap, int sm_count, cudaStream_t st, int* dev_status,
                      unsigned long long* host_stats) {
  if (dist_bits == 32)
    return run_t<uint32_t>(w, g, host_sources, host_o2n, k, bc, width, settle_in, phase_cap, sm_count, st,
                           dev_status, host_stats);
  return run_t<uint64_t>(w, g, host_sources, host_o2n, k, bc, width, settle_in, phase_cap, sm_count, st,
                         dev_status, host_stats);
}

}  // namespace bcgpu
