// The paper's own thread mappings, replayed on GB300 for comparison
// (arxiv 1701.05975, Sec. 3.1-3.4): one source at a time over the whole GPU,
// per phase
//   expand   - node-parallel (Algorithm 2: a group of VW threads for every
//              vertex, work only where F[v] = 1) or work-efficient (Algorithms
//              4-5: groups only for the frontier queue); VW = 1 is one thread
//              per vertex, VW = 4..32 the (virtual) warp-centric mapping of
//              Sec. 3.4;
//   Delta_i  - Eq. 2 over every unsettled reached vertex (a scan of all V);
//   settle   - Eq. 4 over all V (U[v] = 1 and d[v] < Delta_i), appended to S.
// sigma is pulled from predecessors when a vertex is expanded and the
// backward pass follows Algorithm 3 level by level, as in the other paths, so
// the results are exact and identical; only the mapping differs.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "bc_common.h"

namespace bcgpu {
namespace {

constexpr unsigned FULL = 0xffffffffu;

template <typename D>
__device__ __forceinline__ D dinf() {
  return ~D(0);
}
__device__ __forceinline__ uint32_t amin(uint32_t* p, uint32_t v) { return atomicMin(p, v); }
__device__ __forceinline__ uint64_t amin(uint64_t* p, uint64_t v) {
  return (uint64_t)atomicMin(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}
__device__ __forceinline__ uint32_t ldv(const uint32_t* p) { return __ldcg(p); }
__device__ __forceinline__ uint64_t ldv(const uint64_t* p) {
  return (uint64_t)__ldcg(reinterpret_cast<const unsigned long long*>(p));
}

// Lanes of this thread's VW-wide group within its warp.
template <int VW>
__device__ __forceinline__ unsigned group_mask() {
  if constexpr (VW >= 32) {
    return FULL;
  } else {
    return ((1u << VW) - 1u) << ((threadIdx.x & 31u) / VW * VW);
  }
}

template <int VW>
__device__ __forceinline__ double group_sum(double x, unsigned mask) {
  if constexpr (VW >= 32) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
  } else if constexpr (VW > 1) {
#pragma unroll
    for (int o = VW / 2; o > 0; o >>= 1) x += __shfl_xor_sync(mask, x, o, VW);
  }
  return x;
}

struct PaperCtr {
  unsigned long long delta;  // Delta_i
  unsigned int S_len, cnt;
};

__device__ __forceinline__ uint2 entry_at(const GraphDev& g, uint64_t e) {
  if (g.adjp) {
    const uint32_t x = g.adjp[e];
    return make_uint2(x & ((1u << g.col_bits) - 1u), x >> g.col_bits);
  }
  return g.adj[e];
}

// Algorithm 1: U = 1, F = 0, d = INF everywhere; then the source.
template <typename D>
__global__ void p_init(uint32_t n, D* d, uint8_t* U, uint8_t* F, double* sig, uint32_t* S, PaperCtr* c, uint32_t s) {
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    d[v] = dinf<D>();
    U[v] = 1;
    F[v] = 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c->S_len = 1;
    S[0] = s;
  }
}

template <typename D>
__global__ void p_init_source(D* d, uint8_t* U, uint8_t* F, double* sig, uint32_t s) {
  d[s] = 0;
  U[s] = 0;
  F[s] = 1;
  sig[s] = 1.0;
}

// Expansion: groups of VW threads; NODE_PAR walks all V (work where F = 1),
// otherwise the frontier list S[f0, f1).
template <typename D, int VW, bool NODE_PAR>
__global__ void p_expand(GraphDev g, D* d, double* sig, const uint8_t* F, const uint32_t* S, uint32_t f0, uint32_t f1,
                         uint32_t s) {
  const D INF = dinf<D>();
  const uint32_t lane = threadIdx.x % VW;
  const uint64_t grp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) / VW;
  const uint64_t ngrp = ((uint64_t)gridDim.x * blockDim.x) / VW;
  const uint64_t items = NODE_PAR ? g.n : (uint64_t)(f1 - f0);
  const unsigned mask = group_mask<VW>();
  for (uint64_t it = grp; it < items; it += ngrp) {
    uint32_t v;
    if (NODE_PAR) {
      v = (uint32_t)it;
      if (!F[v]) continue;  // the whole group skips together
    } else {
      v = S[f0 + it];
    }
    const D dv = ldv(&d[v]);
    double acc = 0.0;
    for (uint64_t e = g.row_ptr[v] + lane; e < g.row_ptr[v + 1]; e += VW) {
      const uint2 ent = entry_at(g, e);
      const uint32_t u = ent.x;
      const D w = (D)ent.y;
      const D du = ldv(&d[u]);
      if (du != INF && du + w == dv) {
        acc += __ldcg(&sig[u]);
      } else {
        const D nd = dv + w;
        if (nd < du) amin(&d[u], nd);
      }
    }
    acc = group_sum<VW>(acc, mask);
    if (lane == 0 && v != s) sig[v] = acc;
  }
}

// Eq. 2 over every unsettled reached vertex.
template <typename D>
__global__ void p_delta(uint32_t n, const D* d, const uint8_t* U, const uint32_t* dnode, PaperCtr* c) {
  unsigned long long m = ~0ull;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const D dv = ldv(&d[v]);
    if (U[v] && dv != dinf<D>() && dnode[v] != 0xffffffffu) m = min(m, (unsigned long long)dv + dnode[v]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(FULL, m, o));
  if ((threadIdx.x & 31) == 0 && m != ~0ull) atomicMin(&c->delta, m);
}

// Eq. 4 over all V: settle, mark the new frontier, append to S.
template <typename D>
__global__ void p_settle(uint32_t n, const D* d, uint8_t* U, uint8_t* F, uint32_t* S, PaperCtr* c) {
  const unsigned long long delta = c->delta;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    F[v] = 0;
    // an unreached vertex (d = INF) never satisfies Eq. 4, even when Delta_i
    // is infinite (the INF word of 32-bit distances is below Delta's sentinel)
    const D dv = ldv(&d[v]);
    if (U[v] && dv != dinf<D>() && (unsigned long long)dv < delta) {
      U[v] = 0;
      F[v] = 1;
      S[atomicAdd(&c->S_len, 1u)] = v;
      atomicAdd(&c->cnt, 1u);
    }
  }
}

__global__ void p_ctl(PaperCtr* c) {
  c->delta = ~0ull;
  c->cnt = 0;
}

// Algorithm 3 for one level, VW threads per vertex.
template <typename D, int VW>
__global__ void p_backward(GraphDev g, const D* d, double* sig, const uint32_t* S, uint32_t b0, uint32_t b1,
                           double* bc) {
  const D INF = dinf<D>();
  const uint32_t lane = threadIdx.x % VW;
  const uint64_t grp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) / VW;
  const uint64_t ngrp = ((uint64_t)gridDim.x * blockDim.x) / VW;
  const unsigned mask = group_mask<VW>();
  for (uint64_t it = grp; it < (uint64_t)(b1 - b0); it += ngrp) {
    const uint32_t v = S[b0 + it];
    const D dv = d[v];
    double acc = 0.0;
    for (uint64_t e = g.row_ptr[v] + lane; e < g.row_ptr[v + 1]; e += VW) {
      const uint2 ent = entry_at(g, e);
      const D du = d[ent.x];
      if (du != INF && du == dv + (D)ent.y) acc += sig[ent.x];
    }
    acc = group_sum<VW>(acc, mask);
    if (lane == 0) {
      const double sg = sig[v];
      const double delta = sg * acc;
      sig[v] = (1.0 + delta) / sg;
      atomicAdd(&bc[g.n2o ? g.n2o[v] : v], delta);
    }
  }
}

inline int blocks_for(uint64_t threads, int sm_count) {
  uint64_t b = (threads + 255) / 256;
  if (b < 1) b = 1;
  const uint64_t cap = (uint64_t)sm_count * 8;
  return (int)(b > cap ? cap : b);
}

#define PCK(x)                        \
  do {                                \
    cudaError_t e_ = (x);             \
    if (e_ != cudaSuccess) return e_; \
  } while (0)

template <typename D, int VW, bool NP>
cudaError_t run_variant(PaperWork* w, const GraphDev& g, const uint32_t* src, const uint32_t* host_o2n, uint32_t k,
                        double* bc, uint64_t phase_cap, int sms, cudaStream_t st, int* status,
                        unsigned long long* stats) {
  D* d = static_cast<D*>(w->d);
  PaperCtr* c = static_cast<PaperCtr*>(w->ctr);
  PaperCtr* hc = static_cast<PaperCtr*>(w->host_ctr);
  const uint32_t n = g.n;
  *status = DEV_OK;
  for (uint32_t i = 0; i < k; ++i) {
    if (src[i] >= n) {
      *status = DEV_ERR_INVALID;
      return cudaSuccess;
    }
    const uint32_t s = host_o2n ? host_o2n[src[i]] : src[i];
    p_init<D><<<blocks_for(n, sms), 256, 0, st>>>(n, d, w->U, w->F, w->sig, w->S, c, s);
    p_init_source<D><<<1, 1, 0, st>>>(d, w->U, w->F, w->sig, s);
    PCK(cudaGetLastError());
    std::vector<uint32_t> ends = {0, 1};
    uint32_t f0 = 0, f1 = 1;
    uint64_t phases = 0;
    for (;;) {
      const uint64_t items = NP ? n : (f1 - f0);
      p_expand<D, VW, NP><<<blocks_for(items * VW, sms), 256, 0, st>>>(g, d, w->sig, w->F, w->S, f0, f1, s);
      p_ctl<<<1, 1, 0, st>>>(c);
      p_delta<D><<<blocks_for(n, sms), 256, 0, st>>>(n, d, w->U, g.dnode, c);
      p_settle<D><<<blocks_for(n, sms), 256, 0, st>>>(n, d, w->U, w->F, w->S, c);
      PCK(cudaGetLastError());
      PCK(cudaMemcpyAsync(hc, c, sizeof(PaperCtr), cudaMemcpyDeviceToHost, st));
      PCK(cudaStreamSynchronize(st));
      if (hc->cnt == 0) break;  // Delta_i = infinity: nothing left to settle
      ++phases;
      f0 = f1;
      f1 = hc->S_len;
      ends.push_back(f1);
      if (phases > phase_cap) {
        *status = DEV_ERR_TIMEOUT;
        return cudaStreamSynchronize(st);
      }
    }
    // the last batch was expanded above (its sigma is final); backward now
    for (size_t lev = ends.size() - 2; lev >= 1; --lev)
      p_backward<D, VW><<<blocks_for((uint64_t)(ends[lev + 1] - ends[lev]) * VW, sms), 256, 0, st>>>(
          g, d, w->sig, w->S, ends[lev], ends[lev + 1], bc);
    PCK(cudaGetLastError());
    if (stats) {
      stats[STAT_SOURCES] += 1;
      stats[STAT_PHASES] += phases;
      stats[STAT_REACHED] += ends.back();
    }
  }
  return cudaStreamSynchronize(st);
}

template <typename D, bool NP>
cudaError_t dispatch_vw(PaperWork* w, const GraphDev& g, const uint32_t* src, const uint32_t* o2n, uint32_t k,
                        double* bc, uint64_t cap, int sms, cudaStream_t st, int* status, unsigned long long* stats,
                        int vw) {
  switch (vw) {
    case 1: return run_variant<D, 1, NP>(w, g, src, o2n, k, bc, cap, sms, st, status, stats);
    case 4: return run_variant<D, 4, NP>(w, g, src, o2n, k, bc, cap, sms, st, status, stats);
    case 8: return run_variant<D, 8, NP>(w, g, src, o2n, k, bc, cap, sms, st, status, stats);
    case 16: return run_variant<D, 16, NP>(w, g, src, o2n, k, bc, cap, sms, st, status, stats);
    case 32: return run_variant<D, 32, NP>(w, g, src, o2n, k, bc, cap, sms, st, status, stats);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

uint64_t paper_bytes(uint32_t n, int dist_bits) { return (uint64_t)n * ((dist_bits / 8) + 8 + 4 + 2) + 4096; }

PaperWork* paper_create(uint32_t n, int dist_bits, cudaError_t* e) {
  PaperWork* w = new PaperWork();
  w->n = n;
  *e = cudaMalloc(&w->d, (size_t)n * (dist_bits / 8));
  if (*e == cudaSuccess) *e = cudaMalloc(&w->sig, (size_t)n * 8);
  if (*e == cudaSuccess) *e = cudaMalloc(&w->S, (size_t)n * 4);
  if (*e == cudaSuccess) *e = cudaMalloc(&w->U, n);
  if (*e == cudaSuccess) *e = cudaMalloc(&w->F, n);
  if (*e == cudaSuccess) *e = cudaMalloc(&w->ctr, sizeof(PaperCtr));
  if (*e == cudaSuccess) *e = cudaMallocHost(&w->host_ctr, sizeof(PaperCtr));
  if (*e != cudaSuccess) {
    paper_destroy(w);
    return nullptr;
  }
  return w;
}

void paper_destroy(PaperWork* w) {
  if (!w) return;
  cudaFree(w->d);
  cudaFree(w->sig);
  cudaFree(w->S);
  cudaFree(w->U);
  cudaFree(w->F);
  cudaFree(w->ctr);
  if (w->host_ctr) cudaFreeHost(w->host_ctr);
  delete w;
}

cudaError_t paper_run(PaperWork* w, const GraphDev& g, int dist_bits, const uint32_t* host_sources,
                      const uint32_t* host_o2n, uint32_t k, double* bc, bool node_parallel, int vwarp,
                      uint64_t phase_cap, int sm_count, cudaStream_t st, int* status, unsigned long long* stats) {
  if (dist_bits == 32)
    return node_parallel
               ? dispatch_vw<uint32_t, true>(w, g, host_sources, host_o2n, k, bc, phase_cap, sm_count, st, status,
                                             stats, vwarp)
               : dispatch_vw<uint32_t, false>(w, g, host_sources, host_o2n, k, bc, phase_cap, sm_count, st, status,
                                              stats, vwarp);
  return node_parallel ? dispatch_vw<uint64_t, true>(w, g, host_sources, host_o2n, k, bc, phase_cap, sm_count, st,
                                                     status, stats, vwarp)
                       : dispatch_vw<uint64_t, false>(w, g, host_sources, host_o2n, k, bc, phase_cap, sm_count, st,
                                                      status, stats, vwarp);
}

}  // namespace bcgpu
