// Batched Brandes kernel: one team of threads (a warp or a whole CTA) per
// source, many sources in flight, sources pulled from a device counter.
//
// Per source (arxiv 1701.05975):
//   forward  - parallel Dijkstra in settle batches (Sec. 3.2, Algorithm 2 with
//              the work-efficient frontier queue of Algorithms 4-5).  A batch
//              is every candidate u with D(u) < Delta', where Delta' <=
//              Delta_i = min_{u in U} (D(u) + Delta_node(u)) (Eq. 2, strict
//              test of Eq. 4); optionally also every u with
//              D(u) < min_{U} D + Delta_node(u) (strict IN test).  Candidates
//              are split into a near queue (D < split) and a far queue; only
//              the near queue is scanned per phase.  The batches are the
//              levels S / ends of Algorithm 1.
//              sigma(v) is pulled from v's predecessors when v's batch is
//              expanded: they all settled in earlier batches, so their sigma
//              is final.  The same adjacency walk relaxes v's neighbours with
//              atomicMin on the distance word (replacing the per-vertex locks
//              of Sec. 3.2).
//   backward - Algorithm 3: levels in reverse; for w in a level,
//              delta(w) = sigma(w) * sum_{successors v} c(v) with
//              c(v) = (1 + delta(v)) / sigma(v) kept in sigma's slot; delta(w)
//              is added to BC with an FP64 atomic.
// Every CSR walk uses a load-balanced edge-parallel chunk: the team takes up
// to TEAM frontier vertices, scans their degrees and spreads the chunk's edges
// evenly over its threads, so hubs never serialise one thread or warp.
// This header holds the device code; bc_batched.cu instantiates the strict
// schedule and bc_batched_delta.cu the delta-stepping one, so the two compile
// in parallel.  Everything is in an anonymous namespace: each translation unit
// owns its instantiations.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "bc_common.h"

namespace bcgpu {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t NONE = 0xffffffffu;
#ifndef BCGPU_UNROLL
#define BCGPU_UNROLL 4
#endif
constexpr int UNROLL = BCGPU_UNROLL;  // independent edge loads in flight per thread
// Settle stages the next batch's rows in shared memory (BCGPU_STAGE=0: off).
#ifndef BCGPU_STAGE
#define BCGPU_STAGE 1
#endif
// 1024-thread teams run one CTA per SM and take six (measured +1.4% on R-MAT;
// six spills heavily in the smaller teams' register budget)
template <int TEAM>
__host__ __device__ constexpr int unroll_of() {
  return TEAM >= 1024 ? 6 : UNROLL;
}
constexpr int NEAR_REGS = 4;          // near-queue entries per thread kept in registers
// Teams of up to 512 threads also keep near queues of up to NEAR_MID entries
// per thread in registers (one gather pass, one team-wide scan).
constexpr int NEAR_MID = 8;
#ifndef BCGPU_FAR_LEVELS
#define BCGPU_FAR_LEVELS 16
#endif
constexpr uint64_t FAR_LEVELS = BCGPU_FAR_LEVELS;   // the second far level starts FAR_LEVELS split widths out

template <typename D>
__device__ __forceinline__ D dinf() {
  return ~D(0);
}

__device__ __forceinline__ uint32_t ldcg(const uint32_t* p) { return __ldcg(p); }
__device__ __forceinline__ uint64_t ldcg(const uint64_t* p) {
  return (uint64_t)__ldcg(reinterpret_cast<const unsigned long long*>(p));
}
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }

// Gathers of a team's own slab (distances, sigma).  A slab is private to one
// CTA and every read is ordered after the writes it must see by the team's
// barrier, so L1-cacheable loads are valid; BCGPU_GATHER_L1=0 keeps them in L2.
#ifndef BCGPU_GATHER_L1
#define BCGPU_GATHER_L1 0
#endif
template <typename T>
__device__ __forceinline__ T ldg_slab(const T* p) {
#if BCGPU_GATHER_L1
  return *p;
#else
  return ldcg(p);
#endif
}

__device__ __forceinline__ uint32_t atomic_min_d(uint32_t* p, uint32_t v) { return atomicMin(p, v); }
__device__ __forceinline__ uint64_t atomic_min_d(uint64_t* p, uint64_t v) {
  return (uint64_t)atomicMin(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}

// FAR_LEVELS split widths, saturating (a caller may set any width)
__device__ __forceinline__ uint64_t far_span(uint64_t width) {
  return width > ~0ull / FAR_LEVELS ? ~0ull : FAR_LEVELS * width;
}

template <typename D>
__device__ __forceinline__ D sat_add(D a, uint64_t b) {
  uint64_t lim = (uint64_t)dinf<D>() - 1;
  uint64_t aa = (uint64_t)a;
  if (aa >= lim || b >= lim - aa) return (D)lim;
  return (D)(aa + b);
}

template <typename D>
__device__ __forceinline__ D shfl_xor_d(D x, int o) {
  return __shfl_xor_sync(FULL, x, o);
}

template <typename D>
__device__ __forceinline__ D dmin(D a, D b) {
  return a < b ? a : b;
}
template <typename D>
__device__ __forceinline__ D dmax(D a, D b) {
  return a < b ? b : a;
}

// d + Delta_node for the OUT threshold (Eq. 2); a vertex without out-edges
// (Delta_node = UINT32_MAX, only in directed graphs) cannot lower any
// distance, so its term is +infinity.
template <typename D>
__device__ __forceinline__ D out_key(D d, uint32_t dnode) {
  return dnode == 0xffffffffu ? dinf<D>() : (D)(d + (D)dnode);
}

template <typename D, int TEAM>
struct TeamShared {
  uint32_t src_idx;
  uint32_t near_len, far_len, far2_len, S_len, nlev;
  uint32_t pair_len, pair_over;
  int stop;
  D xs;  // every reached vertex whose distance is below xs is settled (the last threshold)
  // strict schedule: per-section SM cycles and queue entries scanned (kept by
  // the team leader in shared memory, out of every thread's registers)
  unsigned long long cyc_expand, cyc_refill, cyc_settle, cyc_back, near_sc, far_sc;
  long long tmark;
  D split, split2;  // near < split <= far < split2 <= far2
  uint32_t off[TEAM + 1];
  uint32_t vtx[TEAM];
  unsigned long long rs[TEAM];
  D dv[TEAM];
  double acc[TEAM];
  double sv[TEAM];
  uint32_t dg[TEAM];     // degree of each chunk vertex
  // chunk vertices walked by one warp each / by the whole team (16-bit
  // indices keep a 1024-thread team's state within 48 KB)
  using Idx = typename std::conditional<(TEAM > 512), uint16_t, uint32_t>::type;
  Idx wlist[TEAM];
  Idx tlist[TEAM];
  uint32_t wnext, nwl, ntl;
  uint32_t staged;  // leading entries of the next batch already in vtx / rs / dg / dv
  // delta-stepping schedule
  uint32_t front_len, def_len, lvl_len, round;
  uint32_t* front_out;
  D bound;
  D red[2 * (TEAM / 32) + 2];
  uint32_t scan[2 * (TEAM / 32 + 1)];
};

template <int TEAM>
__device__ __forceinline__ void team_sync() {
  if constexpr (TEAM == 32) {
    __syncwarp();
  } else {
    __syncthreads();
  }
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Exclusive prefix sum over the team; *total receives the team-wide sum.
// Every thread of the team must call it.
template <int TEAM>
__device__ __forceinline__ uint32_t team_excl_scan(uint32_t x, uint32_t* total, uint32_t* scratch) {
  uint32_t inc = warp_incl_scan(x);
  if constexpr (TEAM == 32) {
    *total = __shfl_sync(FULL, inc, 31);
    return inc - x;
  } else {
    constexpr int NW = TEAM / 32;
    const int w = (threadIdx.x % TEAM) >> 5, lane = threadIdx.x & 31;
    if (lane == 31) scratch[w] = inc;
    __syncthreads();
    if (w == 0) {
      uint32_t v = lane < NW ? scratch[lane] : 0u;
      uint32_t vi = warp_incl_scan(v);
      if (lane < NW) scratch[lane] = vi - v;
      if (lane == NW - 1) scratch[NW] = vi;
    }
    __syncthreads();
    *total = scratch[NW];
    uint32_t r = scratch[w] + inc - x;
    __syncthreads();
    return r;
  }
}

// Two exclusive prefix sums at once (shares the barriers).
template <int TEAM>
__device__ __forceinline__ void team_excl_scan2(uint32_t x, uint32_t y, uint32_t* ex, uint32_t* ey, uint32_t* tx,
                                                uint32_t* ty, uint32_t* scratch) {
  const uint32_t ix = warp_incl_scan(x), iy = warp_incl_scan(y);
  if constexpr (TEAM == 32) {
    *tx = __shfl_sync(FULL, ix, 31);
    *ty = __shfl_sync(FULL, iy, 31);
    *ex = ix - x;
    *ey = iy - y;
  } else {
    constexpr int NW = TEAM / 32;
    const int w = (threadIdx.x % TEAM) >> 5, lane = threadIdx.x & 31;
    if (lane == 31) {
      scratch[w] = ix;
      scratch[NW + 1 + w] = iy;
    }
    __syncthreads();
    if (w == 0) {
      const uint32_t vx = lane < NW ? scratch[lane] : 0u, vy = lane < NW ? scratch[NW + 1 + lane] : 0u;
      const uint32_t sx = warp_incl_scan(vx), sy = warp_incl_scan(vy);
      if (lane < NW) {
        scratch[lane] = sx - vx;
        scratch[NW + 1 + lane] = sy - vy;
      }
      if (lane == NW - 1) {
        scratch[NW] = sx;
        scratch[2 * NW + 1] = sy;
      }
    }
    __syncthreads();
    *tx = scratch[NW];
    *ty = scratch[2 * NW + 1];
    *ex = scratch[w] + ix - x;
    *ey = scratch[NW + 1 + w] + iy - y;
    __syncthreads();
  }
}

// Team-wide minimum of two values at once.
template <typename D, int TEAM>
__device__ __forceinline__ void team_min2(D& a, D& b, D* scratch) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = dmin(a, shfl_xor_d(a, o));
    b = dmin(b, shfl_xor_d(b, o));
  }
  if constexpr (TEAM > 32) {
    constexpr int NW = TEAM / 32;
    const int w = (threadIdx.x % TEAM) >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
      scratch[w] = a;
      scratch[NW + w] = b;
    }
    __syncthreads();
    if (w == 0) {
      D x = lane < NW ? scratch[lane] : dinf<D>();
      D y = lane < NW ? scratch[NW + lane] : dinf<D>();
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        x = dmin(x, shfl_xor_d(x, o));
        y = dmin(y, shfl_xor_d(y, o));
      }
      if (lane == 0) {
        scratch[2 * NW] = x;
        scratch[2 * NW + 1] = y;
      }
    }
    __syncthreads();
    a = scratch[2 * NW];
    b = scratch[2 * NW + 1];
    __syncthreads();
  }
}

// L2 residency hints.  The distance words of the highest-degree vertices (a
// prefix of the ids after relabeling) are gathered by most edges and are
// loaded with an evict-last policy (measured: +2% on R-MAT).  Marking the
// streamed adjacency evict-first measured slower and is off by default.
#ifndef BCGPU_ADJ_HINT
#define BCGPU_ADJ_HINT 0
#endif
#ifndef BCGPU_HOT_HINT
#define BCGPU_HOT_HINT 1
#endif
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// CSR entry e as {neighbour, weight}: from the packed 32-bit form
// (neighbour | weight << col_bits) when PACKED, else from {col, w} records.
// One CSR (the out-edges, or for directed graphs the in-edges) as a walk sees it.
struct Rows {
  const uint64_t* row_ptr;
  const uint2* adj;
  const uint32_t* adjp;
  uint32_t col_bits;
};

__device__ __forceinline__ Rows out_rows(const GraphDev& g) { return Rows{g.row_ptr, g.adj, g.adjp, g.col_bits}; }
__device__ __forceinline__ Rows in_rows(const GraphDev& g) { return Rows{g.in_row_ptr, g.in_adj, g.in_adjp, g.col_bits}; }

template <bool PACKED>
__device__ __forceinline__ uint2 load_entry(const Rows& g, uint64_t e, uint64_t pol) {
#if BCGPU_ADJ_HINT
  if constexpr (PACKED) {
    uint32_t x;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(x) : "l"(g.adjp + e), "l"(pol));
    return make_uint2(x & ((1u << g.col_bits) - 1u), x >> g.col_bits);
  } else {
    uint2 r;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.b32 {%0, %1}, [%2], %3;"
                 : "=r"(r.x), "=r"(r.y) : "l"(g.adj + e), "l"(pol));
    return r;
  }
#else
  (void)pol;
  if constexpr (PACKED) {
    const uint32_t x = __ldg(&g.adjp[e]);
    return make_uint2(x & ((1u << g.col_bits) - 1u), x >> g.col_bits);
  } else {
    return __ldg(&g.adj[e]);
  }
#endif
}

// Distance gather: L2-only load, evict-last for the hot id prefix.
__device__ __forceinline__ uint32_t gather_d(const uint32_t* d, uint32_t u, uint32_t hot_n, uint64_t pol) {
#if BCGPU_HOT_HINT
  if (u < hot_n) {
    uint32_t x;
    asm volatile("ld.global.cg.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(x) : "l"(d + u), "l"(pol));
    return x;
  }
#endif
  return __ldcg(d + u);
}
__device__ __forceinline__ uint64_t gather_d(const uint64_t* d, uint32_t u, uint32_t hot_n, uint64_t pol) {
#if BCGPU_HOT_HINT
  if (u < hot_n) {
    uint64_t x;
    asm volatile("ld.global.cg.L2::cache_hint.b64 %0, [%1], %2;" : "=l"(x) : "l"(d + u), "l"(pol));
    return x;
  }
#endif
  return (uint64_t)__ldcg(reinterpret_cast<const unsigned long long*>(d + u));
}

// Sigma gather of a predecessor: evict-last for the hot id prefix when
// BCGPU_HOT_SIG is set (off by default).
#ifndef BCGPU_HOT_SIG
#define BCGPU_HOT_SIG 0
#endif
__device__ __forceinline__ double gather_sig(const double* s, uint32_t u, uint32_t hot_n, uint64_t pol) {
  if (u < hot_n) {
    double x;
    asm volatile("ld.global.cg.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(x) : "l"(s + u), "l"(pol));
    return x;
  }
  return __ldcg(s + u);
}

template <typename D>
struct Slab {
  D* d;
  double* sig;
  uint32_t* S;
  uint32_t* ends;
  uint32_t* nearq;
  uint32_t* farq;
  uint32_t* farq2;
  double* bacc;     // backward accumulator: sum of successor coefficients
  uint32_t* pend;   // pend[l] = end of level l's DAG edges in pairs
  uint2* pairs;     // DAG edges {predecessor u, vertex v}
  uint32_t pair_cap;
  uint32_t* pc;     // delta-stepping: round stamps, then predecessor counts (zero between sources)
  uint32_t* pair_e; // edge output: the walked entry of each DAG edge, else nullptr
};

template <typename D>
__device__ __forceinline__ Slab<D> slab_at(const BatchArgs& a, uint32_t slot) {
  char* base = a.slabs + (uint64_t)slot * a.lay.stride;
  Slab<D> s;
  s.d = reinterpret_cast<D*>(base + a.lay.off_d);
  s.sig = reinterpret_cast<double*>(base + a.lay.off_sig);
  s.S = reinterpret_cast<uint32_t*>(base + a.lay.off_S);
  s.ends = reinterpret_cast<uint32_t*>(base + a.lay.off_ends);
  s.nearq = reinterpret_cast<uint32_t*>(base + a.lay.off_near);
  s.farq = reinterpret_cast<uint32_t*>(base + a.lay.off_far);
  s.farq2 = reinterpret_cast<uint32_t*>(base + a.lay.off_far2);
  s.bacc = reinterpret_cast<double*>(base + a.lay.off_acc);
  s.pend = reinterpret_cast<uint32_t*>(base + a.lay.off_pend);
  s.pairs = reinterpret_cast<uint2*>(base + a.lay.off_pairs);
  s.pair_cap = a.lay.pair_cap;
  s.pc = reinterpret_cast<uint32_t*>(base + a.lay.off_pc);
  s.pair_e = (a.ebc && a.esm && a.lay.off_pair_e) ? reinterpret_cast<uint32_t*>(base + a.lay.off_pair_e) : nullptr;
  return s;
}

// Load a chunk [base, base + cnt) of a level list into shared memory and scan
// the degrees.  Returns the chunk's edge total (uniform over the team).
template <typename D, int TEAM>
__device__ __forceinline__ uint32_t load_chunk(const BatchArgs& a, const Slab<D>& sl, TeamShared<D, TEAM>& sh,
                                               const uint32_t* list, uint32_t base, uint32_t cnt, int t,
                                               bool want_sigma) {
  uint32_t deg = 0;
  if ((uint32_t)t < cnt) {
    uint32_t v = ldcg(&list[base + t]);
    uint64_t r0 = __ldg(&a.g.row_ptr[v]);
    uint64_t r1 = __ldg(&a.g.row_ptr[v + 1]);
    deg = (uint32_t)(r1 - r0);
    sh.vtx[t] = v;
    sh.rs[t] = r0;
    sh.dv[t] = ldcg(&sl.d[v]);
    sh.acc[t] = 0.0;
    if (want_sigma) sh.sv[t] = ldcg(&sl.sig[v]);
  }
  uint32_t total;
  uint32_t ex = team_excl_scan<TEAM>(deg, &total, sh.scan);
  if ((uint32_t)t < cnt) sh.off[t] = ex;
  if (t == 0) sh.off[cnt] = total;
  team_sync<TEAM>();
  return total;
}

// Index i of the chunk vertex owning chunk edge e: off[i] <= e < off[i + 1].
template <int TEAM>
__device__ __forceinline__ uint32_t owner_of(const uint32_t* off, uint32_t cnt, uint32_t e) {
  uint32_t lo = 0, hi = cnt;
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (off[mid] <= e) lo = mid; else hi = mid;
  }
  return lo;
}

// One CSR entry {u, w} of chunk vertex i during the forward pass: if u is a
// shortest-path predecessor (settled in an earlier batch), pull its sigma and
// record the DAG edge u -> v; otherwise relax u.
// Walk modes: an undirected row serves both the sigma pull and the
// relaxation; a directed graph pulls over its in-edges and relaxes over its
// out-edges in two walks.
// The delta-stepping schedule adds three walks: relaxation into the next
// round's frontier (WALK_DS), counting each vertex's predecessors once the
// distances are final (WALK_COUNT), and pushing sigma down the DAG level by
// level (WALK_KAHN).
enum : int { WALK_BOTH = 0, WALK_PULL = 1, WALK_RELAX = 2, WALK_DS = 3, WALK_COUNT = 4, WALK_KAHN = 5 };

template <typename D, int TEAM, int MODE>
__device__ __forceinline__ void visit_entry(const Slab<D>& sl, TeamShared<D, TEAM>& sh, uint32_t i, uint2 ent, D du,
                                            D split, unsigned long long& relax, uint32_t hot_n, uint64_t pol_last,
                                            uint64_t eidx) {
  (void)hot_n;
  (void)pol_last;
  const D INF = dinf<D>();
  const uint32_t u = ent.x;
  const D w = (D)ent.y;
  const D dvi = sh.dv[i];
  if constexpr (MODE == WALK_DS) {
    const D nd = dvi + w;
    if (nd < du) {
      ++relax;
      const D old = atomic_min_d(&sl.d[u], nd);
      if (nd < old) {
        if (old == INF) sl.S[atomicAdd(&sh.S_len, 1u)] = u;  // reached list
        if (nd < sh.bound) {
          // once per round in the next frontier (stamp = that round)
          if (atomicExch(&sl.pc[u], sh.round) != sh.round) sh.front_out[atomicAdd(&sh.front_len, 1u)] = u;
        } else if (old == INF) {
          sl.farq2[atomicAdd(&sh.def_len, 1u)] = u;  // deferred to a later bucket
        }
      }
    }
    return;
  } else if constexpr (MODE == WALK_COUNT) {
    if (du != INF && du + w == dvi) atomicAdd(&sh.acc[i], 1.0);
    return;
  } else if constexpr (MODE == WALK_KAHN) {
    if (du != INF && du == dvi + w) {
      // u is a successor: push sigma; the last predecessor releases u
      atomicAdd(&sl.sig[u], sh.sv[i]);
      if (atomicSub(&sl.pc[u], 1u) == 1u) sl.ends[atomicAdd(&sh.lvl_len, 1u)] = u;
    }
    return;
  }
  if (MODE != WALK_RELAX && du != INF && du + w == dvi) {
#if BCGPU_HOT_SIG
    atomicAdd(&sh.acc[i], gather_sig(sl.sig, u, hot_n, pol_last));
#else
    atomicAdd(&sh.acc[i], ldg_slab(&sl.sig[u]));
#endif
    const uint32_t pos = atomicAdd(&sh.pair_len, 1u);
    if (pos < sl.pair_cap) {
      sl.pairs[pos] = make_uint2(u, sh.vtx[i]);
      if (sl.pair_e) sl.pair_e[pos] = (uint32_t)eidx;
    } else {
      sh.pair_over = 1;
    }
  } else if (MODE != WALK_PULL) {
    const D nd = dvi + w;
    if (nd < du) {
      ++relax;
      const D old = atomic_min_d(&sl.d[u], nd);
      if (nd < old) {
        // first touch: queue by range; a later drop across a boundary
        // queues u again in the lower range (the older entry goes stale)
        if (nd < split) {
          if (old >= split) sl.nearq[atomicAdd(&sh.near_len, 1u)] = u;
        } else {
          const D split2 = sh.split2;
          if (nd < split2) {
            if (old >= split2) sl.farq[atomicAdd(&sh.far_len, 1u)] = u;
          } else if (old == INF) {
            sl.farq2[atomicAdd(&sh.far2_len, 1u)] = u;
          }
        }
      }
    }
  }
}

// `lanes` threads (this one is number l) walk the whole row of chunk vertex i,
// unroll_of<TEAM>() independent adjacency loads and distance gathers in flight each.
template <typename D, int TEAM, bool PACKED, int MODE>
__device__ __forceinline__ void walk_row(const BatchArgs& a, const Rows& rows, const Slab<D>& sl,
                                         TeamShared<D, TEAM>& sh, uint32_t i, uint32_t l, uint32_t lanes, D split,
                                         unsigned long long& relax) {
  constexpr int UNR = unroll_of<TEAM>();
  const D INF = dinf<D>();
  const uint64_t r0 = sh.rs[i];
  const uint32_t deg = sh.dg[i];
  const uint64_t pf = policy_evict_first(), pl = policy_evict_last();
  for (uint32_t e0 = l; e0 < deg; e0 += lanes * UNR) {
    uint2 ent[UNR];
#pragma unroll
    for (int q = 0; q < UNR; ++q) {
      const uint32_t e = e0 + q * lanes;
      ent[q] = e < deg ? load_entry<PACKED>(rows, r0 + e, pf) : make_uint2(0, 0);
    }
    D dus[UNR];
#pragma unroll
    for (int q = 0; q < UNR; ++q) dus[q] = (e0 + q * lanes < deg) ? gather_d(sl.d, ent[q].x, a.hot_n, pl) : INF;
#pragma unroll
    for (int q = 0; q < UNR; ++q)
      if (e0 + q * lanes < deg)
        visit_entry<D, TEAM, MODE>(sl, sh, i, ent[q], dus[q], split, relax, a.hot_n, pl, r0 + e0 + q * lanes);
  }
}

// Forward expansion of the batch S[f0, f1): sigma pull + relaxation.  Each
// chunk of up to TEAM vertices is split by degree: rows of at least
// team_deg entries are walked by the whole team one after another, rows of
// at least warp_deg entries by one warp each (taken dynamically), and the
// remaining short rows are spread edge by edge over all threads (a degree
// scan plus a binary search for each edge's row).  No barrier separates the
// tiers, so threads that finish one move on to the next.
template <typename D, int TEAM, bool PACKED, int MODE>
__device__ void expand_forward(const BatchArgs& a, const Rows& rows, const Slab<D>& sl, TeamShared<D, TEAM>& sh,
                               const uint32_t* list, uint32_t f0, uint32_t f1, uint32_t s, int t, D split,
                               unsigned long long& relax, unsigned long long& scanned, uint32_t staged = 0) {
  constexpr int UNR = unroll_of<TEAM>();
  const D INF = dinf<D>();
  const uint32_t warp_deg = a.warp_deg;
  const uint32_t team_deg = (TEAM == 32) ? a.warp_deg : a.team_deg;
  for (uint32_t base = f0; base < f1; base += TEAM) {
    const uint32_t cnt = min((uint32_t)TEAM, f1 - base);
    uint32_t deg = 0, small = 0, is_w = 0, is_t = 0;
    if ((uint32_t)t < cnt) {
      if (base == f0 && (uint32_t)t < staged) {
        deg = sh.dg[t];  // placed by the settle step that formed this batch
      } else {
        const uint32_t v = ldcg(&list[base + t]);
        const uint64_t r0 = __ldg(&rows.row_ptr[v]);
        deg = (uint32_t)(__ldg(&rows.row_ptr[v + 1]) - r0);
        sh.vtx[t] = v;
        sh.rs[t] = r0;
        sh.dg[t] = deg;
        sh.dv[t] = ldcg(&sl.d[v]);
      }
      sh.acc[t] = 0.0;
      if (MODE == WALK_KAHN) sh.sv[t] = ldcg(&sl.sig[sh.vtx[t]]);
      if (deg >= team_deg) is_t = 1;
      else if (deg >= warp_deg) is_w = 1;
      else small = deg;
    }
    uint32_t ex_small, ex_tier, total_small, tiers;
    // the tier counts are packed: warp-walked in the low 16 bits, team-walked above
    team_excl_scan2<TEAM>(small, is_w | (is_t << 16), &ex_small, &ex_tier, &total_small, &tiers, sh.scan);
    if ((uint32_t)t < cnt) {
      sh.off[t] = ex_small;
      if (is_w) sh.wlist[ex_tier & 0xffffu] = t;
      if (is_t) sh.tlist[ex_tier >> 16] = t;
    }
    if (t == 0) {
      sh.off[cnt] = total_small;
      sh.wnext = 0;
    }
    team_sync<TEAM>();
    const uint32_t nw = tiers & 0xffffu, nt = tiers >> 16;
    scanned += (t == 0) ? (uint64_t)total_small : 0;
    // tier 3: whole team per row
    for (uint32_t h = 0; h < nt; ++h) {
      const uint32_t i = sh.tlist[h];
      if (t == 0) scanned += sh.dg[i];
      walk_row<D, TEAM, PACKED, MODE>(a, rows, sl, sh, i, (uint32_t)t, TEAM, split, relax);
    }
    // tier 2: one warp per row, rows taken in turn
    if constexpr (TEAM > 32) {
      const uint32_t lane = threadIdx.x & 31;
      for (;;) {
        uint32_t wi = 0;
        if (lane == 0) wi = atomicAdd(&sh.wnext, 1u);
        wi = __shfl_sync(FULL, wi, 0);
        if (wi >= nw) break;
        const uint32_t i = sh.wlist[wi];
        if (lane == 0) scanned += sh.dg[i];
        walk_row<D, TEAM, PACKED, MODE>(a, rows, sl, sh, i, lane, 32, split, relax);
      }
    }
    // tier 1: short rows, edge-parallel over the whole team
    const uint64_t pf = policy_evict_first(), pl = policy_evict_last();
    for (uint32_t e0 = t; e0 < total_small; e0 += TEAM * UNR) {
      uint32_t iv[UNR];
      uint2 ent[UNR];
#pragma unroll
      for (int q = 0; q < UNR; ++q) {
        const uint32_t e = e0 + q * TEAM;
        iv[q] = NONE;
        ent[q] = make_uint2(0, 0);
        if (e < total_small) {
          iv[q] = owner_of<TEAM>(sh.off, cnt, e);
          ent[q] = load_entry<PACKED>(rows, sh.rs[iv[q]] + (e - sh.off[iv[q]]), pf);
        }
      }
      D dus[UNR];
#pragma unroll
      for (int q = 0; q < UNR; ++q) dus[q] = (iv[q] != NONE) ? gather_d(sl.d, ent[q].x, a.hot_n, pl) : INF;
#pragma unroll
      for (int q = 0; q < UNR; ++q)
        if (iv[q] != NONE)
          visit_entry<D, TEAM, MODE>(sl, sh, iv[q], ent[q], dus[q], split, relax, a.hot_n, pl,
                                     sh.rs[iv[q]] + (e0 + q * TEAM - sh.off[iv[q]]));
    }
    team_sync<TEAM>();
    if ((MODE == WALK_BOTH || MODE == WALK_PULL) && (uint32_t)t < cnt && sh.vtx[t] != s)
      sl.sig[sh.vtx[t]] = sh.acc[t];
    if (MODE == WALK_COUNT && (uint32_t)t < cnt) {
      const uint32_t v = sh.vtx[t];
      sl.pc[v] = (uint32_t)sh.acc[t];
      sl.sig[v] = (v == s) ? 1.0 : 0.0;
    }
    team_sync<TEAM>();
  }
}

// Backward (Algorithm 3) over one level S[f0, f1).
template <typename D, int TEAM, bool PACKED>
__device__ void accumulate_level(const BatchArgs& a, const Slab<D>& sl, TeamShared<D, TEAM>& sh,
                                 const uint32_t* list, uint32_t f0, uint32_t f1, uint32_t s, int t,
                                 unsigned long long& scanned) {
  constexpr int UNR = unroll_of<TEAM>();
  const D INF = dinf<D>();
  const bool edges = a.ebc != nullptr;
  for (uint32_t base = f0; base < f1; base += TEAM) {
    const uint32_t cnt = min((uint32_t)TEAM, f1 - base);
    const uint32_t total = load_chunk<D, TEAM>(a, sl, sh, list, base, cnt, t, edges);
    scanned += (t == 0) ? total : 0;
    for (uint32_t e0 = t; e0 < total; e0 += TEAM * UNR) {
      uint32_t iv[UNR];
      uint64_t entry[UNR];
      uint2 ent[UNR];
#pragma unroll
      for (int q = 0; q < UNR; ++q) {
        const uint32_t e = e0 + q * TEAM;
        iv[q] = NONE;
        entry[q] = 0;
        ent[q] = make_uint2(0, 0);
        if (e < total) {
          iv[q] = owner_of<TEAM>(sh.off, cnt, e);
          entry[q] = sh.rs[iv[q]] + (e - sh.off[iv[q]]);
          ent[q] = load_entry<PACKED>(out_rows(a.g), entry[q], policy_evict_first());
        }
      }
      D dus[UNR];
#pragma unroll
      for (int q = 0; q < UNR; ++q) dus[q] = (iv[q] != NONE) ? ldcg(&sl.d[ent[q].x]) : INF;
#pragma unroll
      for (int q = 0; q < UNR; ++q) {
        if (iv[q] == NONE) continue;
        const uint32_t i = iv[q];
        const D du = dus[q];
        if (du != INF && du == sh.dv[i] + (D)ent[q].y) {
          // ent.x is a successor: its coefficient c is final (later level)
          const double cu = ldcg(&sl.sig[ent[q].x]);
          atomicAdd(&sh.acc[i], cu);
          if (edges) atomicAdd(&a.ebc[a.g.e2o ? __ldg(&a.g.e2o[entry[q]]) : entry[q]], sh.sv[i] * cu);
        }
      }
    }
    team_sync<TEAM>();
    if ((uint32_t)t < cnt) {
      const uint32_t v = sh.vtx[t];
      const double sg = ldcg(&sl.sig[v]);
      const double delta = sg * sh.acc[t];
      sl.sig[v] = (1.0 + delta) / sg;
      if (v != s) atomicAdd(&a.bc[a.g.n2o ? __ldg(&a.g.n2o[v]) : v], delta);
    }
    team_sync<TEAM>();
  }
}

// Backward step 1 for one level: every successor has pushed its coefficient
// into bacc, so delta(v) = sigma(v) * bacc(v) is final; store
// c(v) = (1 + delta(v)) / sigma(v) in sigma's slot and add delta(v) to BC.
template <typename D, int TEAM>
__device__ __forceinline__ void finalize_level(const BatchArgs& a, const Slab<D>& sl, uint32_t b0, uint32_t b1,
                                               int t) {
  for (uint32_t j = b0 + t; j < b1; j += TEAM) {
    const uint32_t v = ldcg(&sl.S[j]);
    const double acc = ldcg(&sl.bacc[v]);
    const double sg = ldcg(&sl.sig[v]);
    const double delta = sg * acc;
    sl.sig[v] = (1.0 + delta) / sg;
    if (acc != 0.0) {
      sl.bacc[v] = 0.0;
      atomicAdd(&a.bc[a.g.n2o ? __ldg(&a.g.n2o[v]) : v], delta);
    }
  }
}

// Backward step 2 for one level: each DAG edge u -> v into the level adds
// c(v) to bacc(u) (FP64 atomics; u lies in an earlier level).
template <int TEAM>
__device__ __forceinline__ void push_level_pairs(const uint2* pairs, double* bacc, const double* sig, uint32_t p0,
                                                 uint32_t p1, int t) {
  constexpr int UNR = unroll_of<TEAM>();
  for (uint32_t p = p0 + t; p < p1; p += TEAM * UNR) {
    uint2 pr[UNR];
#pragma unroll
    for (int q = 0; q < UNR; ++q) pr[q] = (p + q * TEAM < p1) ? __ldcg(&pairs[p + q * TEAM]) : make_uint2(NONE, 0);
    double c[UNR];
#pragma unroll
    for (int q = 0; q < UNR; ++q) c[q] = (pr[q].x != NONE) ? __ldcg(&sig[pr[q].y]) : 0.0;
#pragma unroll
    for (int q = 0; q < UNR; ++q)
      if (pr[q].x != NONE) atomicAdd(&bacc[pr[q].x], c[q]);
  }
}

// The same step with edge output: the DAG edge u -> v also adds its share
// sigma(u) * c(v) (u's sigma is still intact: u lies in an earlier level) to
// the output entry esm[walked entry] (Sec. 1's edge BC, per CSR entry).
template <int TEAM>
__device__ __forceinline__ void push_level_pairs_edges(const uint2* pairs, const uint32_t* pair_e,
                                                       const uint32_t* esm, double* bacc, const double* sig,
                                                       double* ebc, uint32_t p0, uint32_t p1, int t) {
  constexpr int UNR = 2;
  for (uint32_t p = p0 + t; p < p1; p += TEAM * UNR) {
    uint2 pr[UNR];
    uint32_t pe[UNR];
#pragma unroll
    for (int q = 0; q < UNR; ++q) {
      const bool ok = p + q * TEAM < p1;
      pr[q] = ok ? __ldcg(&pairs[p + q * TEAM]) : make_uint2(NONE, 0);
      pe[q] = ok ? __ldcg(&pair_e[p + q * TEAM]) : 0u;
    }
    double c[UNR], su[UNR];
    uint32_t tg[UNR];
#pragma unroll
    for (int q = 0; q < UNR; ++q) {
      const bool ok = pr[q].x != NONE;
      c[q] = ok ? __ldcg(&sig[pr[q].y]) : 0.0;
      su[q] = ok ? __ldcg(&sig[pr[q].x]) : 0.0;
      tg[q] = ok ? __ldg(&esm[pe[q]]) : 0u;
    }
#pragma unroll
    for (int q = 0; q < UNR; ++q)
      if (pr[q].x != NONE) {
        atomicAdd(&bacc[pr[q].x], c[q]);
        atomicAdd(&ebc[tg[q]], su[q] * c[q]);
      }
  }
}

// Delta_node(u) (dn), raised to u's second smallest incident weight when u's
// lightest neighbour is known to be settled: its distance is below xs, and
// every reached vertex below xs is settled (xs is the previous phase's
// threshold).  Every edge from u to a vertex still unsettled then weighs at
// least the returned bound, so Eq. 2's minimum over d(u) + bound(u) and the
// IN test with it stay legal (Eq. 4's strict test still keeps every
// predecessor of a settled vertex in an earlier batch) and settle larger
// batches.  Undirected graphs only (a.refine).
template <typename D>
__device__ __forceinline__ uint32_t edge_bound(const BatchArgs& a, const Slab<D>& sl, uint32_t u, uint32_t dn,
                                               D xs) {
  if (a.refine) {
    const uint32_t nb = __ldg(&a.g.dnode_arg[u]);
    if (nb != NONE && ldcg(&sl.d[nb]) < xs) return __ldg(&a.g.dnode2[u]);
  }
  return dn;
}

// Team leader: add the cycles since the last mark to a section counter.
template <typename D, int TEAM>
__device__ __forceinline__ void lap(TeamShared<D, TEAM>& sh, int t, unsigned long long& section) {
  if (t == 0) {
    const long long now = clock64();
    section += (unsigned long long)(now - sh.tmark);
    sh.tmark = now;
  }
}

// Returns false when the source hit the phase cap (its slab is then dirty).
template <typename D, int TEAM, bool PACKED>
__device__ bool run_source(const BatchArgs& a, const Slab<D>& sl, TeamShared<D, TEAM>& sh, uint32_t s, int t) {
  const D INF = dinf<D>();
  unsigned long long relax = 0, scanned = 0;
  uint64_t phases = 0, refills = 0;
  // Algorithm 1 / 4: d = INF everywhere already (slab invariant)
  if (t == 0) {
    sl.d[s] = 0;
    sl.sig[s] = 1.0;
    sl.S[0] = s;
    sl.ends[0] = 0;
    sl.ends[1] = 1;
    sh.near_len = 0;
    sh.far_len = 0;
    sh.far2_len = 0;
    sh.S_len = 1;
    sh.nlev = 1;
    sh.pair_len = 0;
    sh.pair_over = 0;
    sh.stop = 0;
    sh.split = sat_add<D>((D)0, a.width);
    sh.split2 = sat_add<D>((D)0, far_span(a.width));
    sh.staged = 0;
    sh.cyc_expand = sh.cyc_refill = sh.cyc_settle = sh.cyc_back = sh.near_sc = sh.far_sc = 0;
    sh.xs = 1;  // weights are >= 1: only the source lies below 1
  }
  team_sync<TEAM>();
  uint32_t f0 = 0, f1 = 1;
  // undirected graphs walk the out-edge rows once per batch, so the settle
  // step can stage the new batch's rows for the next expansion
  const bool stage = BCGPU_STAGE && a.g.in_row_ptr == nullptr;
  for (;;) {
    const D split0 = sh.split;
    if (t == 0) sh.tmark = clock64();
    if (a.g.in_row_ptr) {
      // directed: sigma from in-edges, then relax out-edges
      expand_forward<D, TEAM, PACKED, WALK_PULL>(a, in_rows(a.g), sl, sh, sl.S, f0, f1, s, t, split0, relax,
                                                  scanned);
      expand_forward<D, TEAM, PACKED, WALK_RELAX>(a, out_rows(a.g), sl, sh, sl.S, f0, f1, s, t, split0, relax,
                                                   scanned);
    } else {
      expand_forward<D, TEAM, PACKED, WALK_BOTH>(a, out_rows(a.g), sl, sh, sl.S, f0, f1, s, t, split0, relax,
                                                  scanned, sh.staged);
    }
    // DAG edges into the batch just expanded end here
    if (t == 0) sl.pend[sh.nlev - 1] = sh.pair_len;
    lap(sh, t, sh.cyc_expand);
    // refill the near queue from the far queue when it runs dry, and the far
    // queue from the second far level when that runs dry too
    while (sh.near_len == 0 && (sh.far_len > 0 || sh.far2_len > 0)) {
      if (sh.far_len == 0) {
        // every vertex below split2 is settled: split moves up to split2
        const D old2 = sh.split2;
        const uint32_t fl2 = sh.far2_len;
        if (t == 0) sh.far_sc += 2ull * fl2;
        D lo = INF, dummy = INF;
        for (uint32_t base = 0; base < fl2; base += TEAM) {
          const uint32_t j = base + t;
          if (j < fl2) {
            const D du = ldcg(&sl.d[ldcg(&sl.farq2[j])]);
            if (du >= old2) lo = dmin(lo, du);
          }
        }
        team_min2<D, TEAM>(lo, dummy, sh.red);
        const D ns2 = (lo == INF) ? old2 : sat_add<D>(lo, far_span(a.width));
        uint32_t kept = 0;
        for (uint32_t base = 0; base < fl2; base += TEAM) {
          const uint32_t j = base + t;
          uint32_t u = 0, keep = 0;
          if (j < fl2) {
            u = ldcg(&sl.farq2[j]);
            const D du = ldcg(&sl.d[u]);
            if (du >= old2) {  // below old2: queued again in a lower range already
              if (du < ns2) sl.farq[atomicAdd(&sh.far_len, 1u)] = u;
              else keep = 1;
            }
          }
          uint32_t ktot;
          const uint32_t kx = team_excl_scan<TEAM>(keep, &ktot, sh.scan);
          if (TEAM == 32) __syncwarp();
          if (keep) sl.farq2[kept + kx] = u;
          kept += ktot;
        }
        team_sync<TEAM>();
        if (t == 0) {
          sh.far2_len = kept;
          sh.split = old2;
          sh.split2 = ns2;
        }
        ++refills;
        team_sync<TEAM>();
        continue;
      }
      const D old = sh.split;
      const D cap = sh.split2;
      const uint32_t fl = sh.far_len;
      if (t == 0) sh.far_sc += 2ull * fl;
      D lo = INF, dummy = INF;
      for (uint32_t base = 0; base < fl; base += TEAM) {
        const uint32_t j = base + t;
        if (j < fl) {
          const D du = ldcg(&sl.d[ldcg(&sl.farq[j])]);
          if (du >= old) lo = dmin(lo, du);
        }
      }
      team_min2<D, TEAM>(lo, dummy, sh.red);
      const D ns = (lo == INF) ? old : dmin(sat_add<D>(lo, a.width), cap);
      uint32_t kept = 0;
      for (uint32_t base = 0; base < fl; base += TEAM) {
        const uint32_t j = base + t;
        uint32_t u = 0, keep = 0;
        if (j < fl) {
          u = ldcg(&sl.farq[j]);
          const D du = ldcg(&sl.d[u]);
          if (du >= old) {  // below the old split: already handled by the near queue
            if (du < ns) {
              sl.nearq[atomicAdd(&sh.near_len, 1u)] = u;
            } else {
              keep = 1;
            }
          }
        }
        uint32_t ktot;
        const uint32_t kx = team_excl_scan<TEAM>(keep, &ktot, sh.scan);
        if (TEAM == 32) __syncwarp();
        if (keep) sl.farq[kept + kx] = u;
        kept += ktot;
      }
      team_sync<TEAM>();
      if (t == 0) {
        sh.far_len = kept;
        sh.split = ns;
      }
      ++refills;
      if (phases + refills > a.phase_cap && t == 0) sh.stop = DEV_ERR_TIMEOUT;
      team_sync<TEAM>();
      if (sh.stop) break;
    }
    lap(sh, t, sh.cyc_refill);
    if (sh.stop || sh.near_len == 0) break;
    // threshold: Delta' = min(min_near (D + Delta_node), split) <= Delta_i
    const uint32_t nl = sh.near_len;
    const D split = sh.split;
    const D xs = sh.xs;
    const uint32_t S0 = sh.S_len;
    uint32_t nset = 0, kept = 0;
    D thr_used = 0;
    bool staged_now = false;
    if (nl <= TEAM * NEAR_REGS) {
      staged_now = stage;
      // the whole near queue fits in registers: one gather pass
      if (t == 0) sh.near_sc += nl;
      uint32_t uu[NEAR_REGS];
      D dd[NEAR_REGS], dn[NEAR_REGS], dni[NEAR_REGS];
      D out = INF, dm = INF;
#pragma unroll
      for (int r = 0; r < NEAR_REGS; ++r) {
        const uint32_t j = r * TEAM + t;
        uu[r] = 0;
        dd[r] = INF;
        dn[r] = 0;
        dni[r] = 0;
        if (j < nl) {
          uu[r] = ldcg(&sl.nearq[j]);
          dd[r] = ldcg(&sl.d[uu[r]]);
          dn[r] = (D)edge_bound<D>(a, sl, uu[r], __ldg(&a.g.dnode[uu[r]]), xs);
          dni[r] = a.g.dnode_in ? (D)__ldg(&a.g.dnode_in[uu[r]]) : dn[r];
          out = dmin(out, out_key<D>(dd[r], (uint32_t)dn[r]));
          dm = dmin(dm, dd[r]);
        }
      }
      team_min2<D, TEAM>(out, dm, sh.red);
      const D thr = dmin(out, split);
      thr_used = thr;
#pragma unroll
      for (int r = 0; r < NEAR_REGS; ++r) {
        const uint32_t base = r * TEAM;
        if (base >= nl) break;  // uniform over the team
        const uint32_t j = base + t;
        const uint32_t valid = j < nl;
        uint32_t take = valid && dd[r] < thr;
        if (valid && a.settle_in && !take) take = dd[r] < (D)(dm + dni[r]);
        // the row bounds of a settling vertex load while the scan's barriers run
        uint64_t rp0 = 0, rp1 = 0;
        if (stage && take) {
          rp0 = __ldg(&a.g.row_ptr[uu[r]]);
          rp1 = __ldg(&a.g.row_ptr[uu[r] + 1]);
        }
        uint32_t stot;
        const uint32_t sx = team_excl_scan<TEAM>(take, &stot, sh.scan);
        if (take) {
          const uint32_t idx = nset + sx;
          sl.S[S0 + idx] = uu[r];
          if (stage && idx < (uint32_t)TEAM) {
            // the next expansion's first chunk: id, final distance, row
            sh.vtx[idx] = uu[r];
            sh.rs[idx] = rp0;
            sh.dg[idx] = (uint32_t)(rp1 - rp0);
            sh.dv[idx] = dd[r];
          }
        }
        if (valid && !take) sl.nearq[kept + (j - base) - sx] = uu[r];
        nset += stot;
        kept += min((uint32_t)TEAM, nl - base) - stot;
      }
    } else if (TEAM <= 512 && nl <= TEAM * NEAR_MID) {
      // a mid-sized near queue: one gather pass into registers, then the
      // whole settle and compaction behind a single team-wide scan of each
      // thread's take / keep counts (the order inside a batch and inside the
      // near queue is free); the IN test's minimum incoming weight is read
      // only for directed graphs, where it differs from Delta_node
      if (t == 0) sh.near_sc += nl;
      uint32_t uu[NEAR_MID], dn[NEAR_MID];
      D dd[NEAR_MID];
      D out = INF, dm = INF;
#pragma unroll
      for (int r = 0; r < NEAR_MID; ++r) {
        const uint32_t j = r * TEAM + t;
        uu[r] = 0;
        dd[r] = INF;
        dn[r] = 0;
        if (j < nl) {
          uu[r] = ldcg(&sl.nearq[j]);
          dd[r] = ldcg(&sl.d[uu[r]]);
          dn[r] = edge_bound<D>(a, sl, uu[r], __ldg(&a.g.dnode[uu[r]]), xs);
          out = dmin(out, out_key<D>(dd[r], dn[r]));
          dm = dmin(dm, dd[r]);
        }
      }
      team_min2<D, TEAM>(out, dm, sh.red);
      const D thr = dmin(out, split);
      thr_used = thr;
      uint32_t tmask = 0, ntake = 0, nkeep = 0;
#pragma unroll
      for (int r = 0; r < NEAR_MID; ++r) {
        if (r * TEAM + t < nl) {
          bool take = dd[r] < thr;
          if (a.settle_in && !take) {
            const D dni = a.g.dnode_in ? (D)__ldg(&a.g.dnode_in[uu[r]]) : (D)dn[r];
            take = dd[r] < (D)(dm + dni);
          }
          if (take) {
            tmask |= 1u << r;
            ++ntake;
          } else {
            ++nkeep;
          }
        }
      }
      uint32_t sx, kx, stot, ktot;
      team_excl_scan2<TEAM>(ntake, nkeep, &sx, &kx, &stot, &ktot, sh.scan);
#pragma unroll
      for (int r = 0; r < NEAR_MID; ++r) {
        if (r * TEAM + t < nl) {
          if ((tmask >> r) & 1u) sl.S[S0 + sx++] = uu[r];
          else sl.nearq[kx++] = uu[r];
        }
      }
      nset = stot;
      kept = ktot;
    } else {
      if (t == 0) sh.near_sc += 2ull * nl;
      D out = INF, dm = INF;
      for (uint32_t base = 0; base < nl; base += TEAM) {
        const uint32_t j = base + t;
        if (j < nl) {
          const uint32_t u = ldcg(&sl.nearq[j]);
          const D du = ldcg(&sl.d[u]);
          out = dmin(out, out_key<D>(du, edge_bound<D>(a, sl, u, __ldg(&a.g.dnode[u]), xs)));
          dm = dmin(dm, du);
        }
      }
      team_min2<D, TEAM>(out, dm, sh.red);
      const D thr = dmin(out, split);
      thr_used = thr;
      // settle (strict) and compact the near queue in place
      for (uint32_t base = 0; base < nl; base += TEAM) {
        const uint32_t j = base + t;
        uint32_t u = 0, take = 0, valid = j < nl;
        if (valid) {
          u = ldcg(&sl.nearq[j]);
          const D du = ldcg(&sl.d[u]);
          take = du < thr;
          if (a.settle_in && !take)
            take = du < (D)(dm + (D)(a.g.dnode_in ? __ldg(&a.g.dnode_in[u])
                                                  : edge_bound<D>(a, sl, u, __ldg(&a.g.dnode[u]), xs)));
        }
        uint32_t stot;
        const uint32_t sx = team_excl_scan<TEAM>(take, &stot, sh.scan);
        if (TEAM == 32) __syncwarp();
        if (take) sl.S[S0 + nset + sx] = u;
        if (valid && !take) sl.nearq[kept + (j - base) - sx] = u;
        const uint32_t ccount = min((uint32_t)TEAM, nl - base);
        nset += stot;
        kept += ccount - stot;
      }
    }
    ++phases;
    team_sync<TEAM>();
    if (t == 0) {
      sh.near_len = kept;
      sh.S_len = S0 + nset;
      sh.staged = staged_now ? min(nset, (uint32_t)TEAM) : 0u;
      if (nset == 0) {
        // every phase settles the smallest candidate (its d is below both
        // d + Delta_node and the split); a phase that settles nothing means
        // an input outside the contract (an asymmetric "undirected" CSR):
        // stop before the level arrays could outgrow n + 2 entries
        sh.stop = DEV_ERR_INTERNAL;
      } else {
        sh.nlev += 1;
        sl.ends[sh.nlev] = S0 + nset;
        if (phases + refills > a.phase_cap) sh.stop = DEV_ERR_TIMEOUT;
      }
      // every vertex still unsettled now has d >= thr: the ones left in the
      // queues failed the test, and a relaxation from a settled u gives at
      // least d(u) + bound(u) >= thr
      sh.xs = dmax(sh.xs, thr_used);
    }
    lap(sh, t, sh.cyc_settle);
    team_sync<TEAM>();
    if (sh.stop) break;
    f0 = S0;
    f1 = S0 + nset;
  }
  const bool failed = sh.stop != 0;
  if (failed) {
    if (t == 0) atomicCAS(a.err, DEV_OK, sh.stop);
    // every touched vertex is settled (S), near or far: restore d = INF there
    const uint32_t sl_n = sh.S_len, nl_n = sh.near_len, fl_n = sh.far_len, fl2_n = sh.far2_len;
    for (uint32_t j = t; j < sl_n; j += TEAM) sl.d[ldcg(&sl.S[j])] = INF;
    for (uint32_t j = t; j < nl_n; j += TEAM) sl.d[ldcg(&sl.nearq[j])] = INF;
    for (uint32_t j = t; j < fl_n; j += TEAM) sl.d[ldcg(&sl.farq[j])] = INF;
    for (uint32_t j = t; j < fl2_n; j += TEAM) sl.d[ldcg(&sl.farq2[j])] = INF;
  } else if (a.flags & RUN_FORWARD_ONLY) {
    if (t == 0 && a.debug_out) {
      a.debug_out[0] = sh.nlev;
      a.debug_out[1] = sh.S_len;
    }
  } else {
    const uint32_t nlev = sh.nlev;
    if (t == 0) sh.tmark = clock64();
    if ((!a.ebc || sl.pair_e) && !sh.pair_over) {
      // Algorithm 3 over the recorded DAG edges: levels in reverse; finalize
      // the level's vertices, then push their coefficients to predecessors
      for (int lev = (int)nlev - 1; lev >= 1; --lev) {
        finalize_level<D, TEAM>(a, sl, ldcg(&sl.ends[lev]), ldcg(&sl.ends[lev + 1]), t);
        team_sync<TEAM>();
        if (sl.pair_e)
          push_level_pairs_edges<TEAM>(sl.pairs, sl.pair_e, a.esm, sl.bacc, sl.sig, a.ebc, ldcg(&sl.pend[lev - 1]),
                                       ldcg(&sl.pend[lev]), t);
        else
          push_level_pairs<TEAM>(sl.pairs, sl.bacc, sl.sig, ldcg(&sl.pend[lev - 1]), ldcg(&sl.pend[lev]), t);
        team_sync<TEAM>();
      }
      if (t == 0) sl.bacc[s] = 0.0;  // the source collected shares it does not keep
    } else {
      // per-entry scan: level 0 is the source; delta(s) is not part of BC,
      // but with edge output its outgoing shortest-path edges carry shares
      const int last = a.ebc ? 0 : 1;
      for (int lev = (int)nlev - 1; lev >= last; --lev) {
        const uint32_t b0 = ldcg(&sl.ends[lev]);
        const uint32_t b1 = ldcg(&sl.ends[lev + 1]);
        accumulate_level<D, TEAM, PACKED>(a, sl, sh, sl.S, b0, b1, s, t, scanned);
      }
    }
    lap(sh, t, sh.cyc_back);
    // restore the slab invariant: d = INF on every vertex this source reached
    const uint32_t n_reached = sh.S_len;
    for (uint32_t j = t; j < n_reached; j += TEAM) sl.d[ldcg(&sl.S[j])] = INF;
  }
  if (a.stats) {
    // relax and scanned are per thread; the rest are uniform (counted once)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      relax += __shfl_xor_sync(FULL, relax, o);
      scanned += __shfl_xor_sync(FULL, scanned, o);
    }
    if ((t & 31) == 0) {
      atomicAdd(&a.stats[STAT_RELAX], relax);
      atomicAdd(&a.stats[STAT_ENTRIES], scanned);
    }
    if (t == 0) {
      atomicAdd(&a.stats[STAT_SOURCES], 1ull);
      atomicAdd(&a.stats[STAT_PHASES], (unsigned long long)phases);
      atomicAdd(&a.stats[STAT_REFILLS], (unsigned long long)refills);
      atomicAdd(&a.stats[STAT_REACHED], (unsigned long long)sh.S_len);
      atomicAdd(&a.stats[STAT_DAG_EDGES], (unsigned long long)sh.pair_len);
      atomicAdd(&a.stats[STAT_LEVELS], (unsigned long long)sh.nlev);
      atomicAdd(&a.stats[STAT_PAIR_OVERFLOW], (unsigned long long)sh.pair_over);
      atomicAdd(&a.stats[STAT_CYC_EXPAND], sh.cyc_expand);
      atomicAdd(&a.stats[STAT_CYC_REFILL], sh.cyc_refill);
      atomicAdd(&a.stats[STAT_CYC_SETTLE], sh.cyc_settle);
      atomicAdd(&a.stats[STAT_CYC_BACKWARD], sh.cyc_back);
      atomicAdd(&a.stats[STAT_NEAR_SCANNED], sh.near_sc);
      atomicAdd(&a.stats[STAT_FAR_SCANNED], sh.far_sc);
    }
  }
  team_sync<TEAM>();
  return !failed;
}


// Delta-stepping schedule (ALGO_DELTA), for graphs whose strict settle batches
// are many and small (high diameter):
//   1. exact distances by delta-stepping rounds: the frontier relaxes its
//      out-edges; improved vertices below the bucket bound form the next
//      round's frontier (each at most once per round), the rest wait in a
//      deferred list until the bound advances;
//   2. one walk counts each reached vertex's shortest-path predecessors;
//   3. sigma is pushed down the shortest-path DAG level by level (Kahn's
//      order): a vertex joins the next level when its last predecessor has
//      pushed to it, so a level holds vertices of equal DAG hop depth and no
//      DAG edge lies inside a level (FP64 atomic sums of integer counts are
//      exact below 2^53);
//   4. Algorithm 3 over those levels in reverse (pull from successors).
// Returns false on a cap hit or a failed consistency check (slab restored).
template <typename D, int TEAM, bool PACKED>
__device__ bool run_source_ds(const BatchArgs& a, const Slab<D>& sl, TeamShared<D, TEAM>& sh, uint32_t s, int t) {
  const D INF = dinf<D>();
  unsigned long long relax = 0, scanned = 0;
  uint64_t rounds = 0, advances = 0;
  unsigned long long cyc_expand = 0, cyc_refill = 0, cyc_settle = 0, cyc_back = 0, far_sc = 0;
  long long c0 = clock64();
  uint32_t* qa = sl.nearq;  // current frontier (stamp = sh.round)
  uint32_t* qb = sl.farq;   // next frontier
  if (t == 0) {
    sl.d[s] = 0;
    sl.S[0] = s;
    sh.S_len = 1;
    qa[0] = s;
    sl.pc[s] = 1;
    sh.round = 1;
    sh.def_len = 0;
    sh.bound = sat_add<D>((D)0, a.width);
    sh.stop = 0;
  }
  team_sync<TEAM>();
  uint32_t alen = 1;
  int err = DEV_OK;
  for (;;) {
    c0 = clock64();
    team_sync<TEAM>();  // every thread has read the last frontier length
    if (t == 0) {
      sh.front_out = qb;
      sh.front_len = 0;
      sh.round += 1;
    }
    team_sync<TEAM>();
    expand_forward<D, TEAM, PACKED, WALK_DS>(a, out_rows(a.g), sl, sh, qa, 0, alen, s, t, INF, relax, scanned);
    cyc_expand += clock64() - c0;
    ++rounds;
    alen = sh.front_len;
    uint32_t* tmp = qa;
    qa = qb;
    qb = tmp;
    if (alen == 0) {
      c0 = clock64();
      // next bucket: the deferred vertices within one width of the smallest
      while (alen == 0 && sh.def_len > 0) {
        const D old = sh.bound;
        const uint32_t dl = sh.def_len;
        far_sc += 2ull * dl;
        D lo = INF, dummy = INF;
        for (uint32_t base = 0; base < dl; base += TEAM) {
          const uint32_t j = base + t;
          if (j < dl) {
            const D du = ldcg(&sl.d[ldcg(&sl.farq2[j])]);
            if (du >= old) lo = dmin(lo, du);
          }
        }
        team_min2<D, TEAM>(lo, dummy, sh.red);
        const D nb = (lo == INF) ? old : sat_add<D>(lo, a.width);
        if (t == 0) sh.front_len = 0;
        team_sync<TEAM>();
        uint32_t kept = 0;
        for (uint32_t base = 0; base < dl; base += TEAM) {
          const uint32_t j = base + t;
          uint32_t u = 0, keep = 0;
          if (j < dl) {
            u = ldcg(&sl.farq2[j]);
            const D du = ldcg(&sl.d[u]);
            if (du >= old) {  // below old: already relaxed in an earlier bucket
              if (du < nb) {
                if (atomicExch(&sl.pc[u], sh.round) != sh.round) qa[atomicAdd(&sh.front_len, 1u)] = u;
              } else {
                keep = 1;
              }
            }
          }
          uint32_t ktot;
          const uint32_t kx = team_excl_scan<TEAM>(keep, &ktot, sh.scan);
          if (TEAM == 32) __syncwarp();
          if (keep) sl.farq2[kept + kx] = u;
          kept += ktot;
        }
        team_sync<TEAM>();
        if (t == 0) {
          sh.def_len = kept;
          sh.bound = nb;
        }
        ++advances;
        team_sync<TEAM>();
        alen = sh.front_len;
      }
      cyc_refill += clock64() - c0;
      if (alen == 0) break;
    }
    if (rounds + advances > a.phase_cap) {
      err = DEV_ERR_TIMEOUT;
      break;
    }
  }
  uint32_t nlev = 0;
  const uint32_t nr = sh.S_len;
  if (err == DEV_OK) {
    // distances are final: count predecessors (in-edges for directed graphs)
    c0 = clock64();
    const Rows prow = a.g.in_row_ptr ? in_rows(a.g) : out_rows(a.g);
    expand_forward<D, TEAM, PACKED, WALK_COUNT>(a, prow, sl, sh, sl.S, 0, nr, s, t, INF, relax, scanned);
    // sigma down the DAG, one hop-depth level at a time
    if (t == 0) {
      sl.ends[0] = s;
      sh.lvl_len = 1;
      sl.pend[0] = 0;
      sl.pend[1] = 1;
    }
    team_sync<TEAM>();
    nlev = 1;
    uint32_t l0 = 0, l1 = 1;
    for (;;) {
      expand_forward<D, TEAM, PACKED, WALK_KAHN>(a, out_rows(a.g), sl, sh, sl.ends, l0, l1, s, t, INF, relax,
                                                 scanned);
      const uint32_t l2 = sh.lvl_len;
      if (l2 == l1) break;
      if (t == 0) sl.pend[nlev + 1] = l2;
      ++nlev;
      l0 = l1;
      l1 = l2;
    }
    team_sync<TEAM>();
    cyc_settle += clock64() - c0;
    if (l1 != nr) err = DEV_ERR_INTERNAL;  // every reached vertex must be released exactly once
  }
  if (err != DEV_OK) {
    if (t == 0) atomicCAS(a.err, DEV_OK, err);
    for (uint32_t j = t; j < nr; j += TEAM) {
      const uint32_t v = ldcg(&sl.S[j]);
      sl.d[v] = INF;
      sl.pc[v] = 0;
    }
  } else if (a.flags & RUN_FORWARD_ONLY) {
    // test hook: present the levels in the S / ends layout of the strict schedule
    for (uint32_t j = t; j < nr; j += TEAM) sl.S[j] = ldcg(&sl.ends[j]);
    team_sync<TEAM>();
    for (uint32_t l = t; l <= nlev; l += TEAM) sl.ends[l] = ldcg(&sl.pend[l]);
    if (t == 0 && a.debug_out) {
      a.debug_out[0] = nlev;
      a.debug_out[1] = nr;
    }
  } else {
    c0 = clock64();
    const int last = a.ebc ? 0 : 1;
    for (int lev = (int)nlev - 1; lev >= last; --lev) {
      const uint32_t b0 = ldcg(&sl.pend[lev]);
      const uint32_t b1 = ldcg(&sl.pend[lev + 1]);
      accumulate_level<D, TEAM, PACKED>(a, sl, sh, sl.ends, b0, b1, s, t, scanned);
    }
    cyc_back += clock64() - c0;
    for (uint32_t j = t; j < nr; j += TEAM) sl.d[ldcg(&sl.S[j])] = INF;
  }
  if (a.stats) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      relax += __shfl_xor_sync(FULL, relax, o);
      scanned += __shfl_xor_sync(FULL, scanned, o);
    }
    if ((t & 31) == 0) {
      atomicAdd(&a.stats[STAT_RELAX], relax);
      atomicAdd(&a.stats[STAT_ENTRIES], scanned);
    }
    if (t == 0) {
      atomicAdd(&a.stats[STAT_SOURCES], 1ull);
      atomicAdd(&a.stats[STAT_PHASES], (unsigned long long)rounds);
      atomicAdd(&a.stats[STAT_REFILLS], (unsigned long long)advances);
      atomicAdd(&a.stats[STAT_REACHED], (unsigned long long)nr);
      atomicAdd(&a.stats[STAT_LEVELS], (unsigned long long)nlev);
      atomicAdd(&a.stats[STAT_CYC_EXPAND], cyc_expand);
      atomicAdd(&a.stats[STAT_CYC_REFILL], cyc_refill);
      atomicAdd(&a.stats[STAT_CYC_SETTLE], cyc_settle);
      atomicAdd(&a.stats[STAT_CYC_BACKWARD], cyc_back);
      atomicAdd(&a.stats[STAT_FAR_SCANNED], far_sc);
    }
  }
  team_sync<TEAM>();
  return err == DEV_OK;
}

// Resident CTAs per SM that a CTA team's register budget is compiled for:
// 64 registers per thread (2048 threads per SM for 32-bit distances; 7/8 of
// that for 64-bit ones, where 64 registers would spill).  Measured with
// -Xptxas -v: naming only the block size let the compiler settle on 56-64
// registers with 24-536 bytes of spills per thread in every CTA-team variant;
// with the residency stated, the 32-bit variants up to 512 threads use 64
// registers and no spills.  Warp teams keep the compiler's choice.
template <typename D, int TEAM, int BLOCK>
__host__ __device__ constexpr int min_blocks_of() {
  return TEAM == 32 ? 1 : (sizeof(D) == 4 ? 1024 / BLOCK : (BLOCK <= 256 ? 896 / BLOCK : 1024 / BLOCK));
}

// One instantiation per schedule, so the strict schedule's register allocation
// does not pay for the delta-stepping code.
template <typename D, int TEAM, int BLOCK, bool PACKED, int ALGO>
__global__ void __launch_bounds__(BLOCK, (min_blocks_of<D, TEAM, BLOCK>())) bc_batched_kernel(const BatchArgs a) {
  static_assert(TEAM == 32 || TEAM == BLOCK, "a CTA holds either warp teams or one team");
  constexpr int NTEAMS = BLOCK / TEAM;
  __shared__ TeamShared<D, TEAM> shared_teams[NTEAMS];
  const int team = threadIdx.x / TEAM;
  const int t = threadIdx.x % TEAM;
  const uint32_t slot = blockIdx.x * NTEAMS + team;
  if (slot >= a.nslots) return;  // a whole team leaves together
  TeamShared<D, TEAM>& sh = shared_teams[team];
  const Slab<D> sl = slab_at<D>(a, slot);
  for (;;) {
    if (t == 0) sh.src_idx = atomicAdd(a.counter, 1u);
    team_sync<TEAM>();
    const uint32_t idx = sh.src_idx;
    team_sync<TEAM>();
    if (idx >= a.k) break;
    uint32_t s = __ldg(&a.sources[idx]);
    if (s >= a.g.n) {
      if (t == 0) atomicCAS(a.err, DEV_OK, DEV_ERR_INVALID);
      continue;
    }
    if (a.g.o2n) s = __ldg(&a.g.o2n[s]);
    bool ok;
    if constexpr (ALGO == ALGO_DELTA)
      ok = run_source_ds<D, TEAM, PACKED>(a, sl, sh, s, t);
    else
      ok = run_source<D, TEAM, PACKED>(a, sl, sh, s, t);
    if (!ok || (a.flags & RUN_FORWARD_ONLY)) break;
  }
}

template <typename D, int TEAM, int BLOCK, bool PACKED, int ALGO>
cudaError_t launch_t(const BatchArgs& a, int grid, cudaStream_t st) {
  bc_batched_kernel<D, TEAM, BLOCK, PACKED, ALGO><<<grid, BLOCK, 0, st>>>(a);
  return cudaGetLastError();
}

// 1024-thread teams exist for 32-bit distances only (their shared state fits
// the 48 KB of static shared memory; 64-bit distance words do not).
template <typename D, bool PACKED, int ALGO>
cudaError_t launch_d(const BatchArgs& a, int team, int grid, cudaStream_t st) {
  switch (team) {
    case 32: return launch_t<D, 32, 256, PACKED, ALGO>(a, grid, st);
    case 128: return launch_t<D, 128, 128, PACKED, ALGO>(a, grid, st);
    case 256: return launch_t<D, 256, 256, PACKED, ALGO>(a, grid, st);
    case 512: return launch_t<D, 512, 512, PACKED, ALGO>(a, grid, st);
    case 1024:
      if constexpr (sizeof(D) == 4) return launch_t<D, 1024, 1024, PACKED, ALGO>(a, grid, st);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

template <typename D, bool PACKED, int ALGO>
cudaError_t occ_d(int team, int* out) {
  switch (team) {
    case 32: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, bc_batched_kernel<D, 32, 256, PACKED, ALGO>, 256, 0);
    case 128: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, bc_batched_kernel<D, 128, 128, PACKED, ALGO>, 128, 0);
    case 256: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, bc_batched_kernel<D, 256, 256, PACKED, ALGO>, 256, 0);
    case 512: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, bc_batched_kernel<D, 512, 512, PACKED, ALGO>, 512, 0);
    case 1024:
      if constexpr (sizeof(D) == 4)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, bc_batched_kernel<D, 1024, 1024, PACKED, ALGO>, 1024, 0);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

// Packed adjacency is only generated for graphs with 32-bit distances.
template <int ALGO>
cudaError_t launch_algo(const BatchArgs& a, int dist_bits, int team, int grid, cudaStream_t st) {
  if (grid <= 0) return cudaSuccess;
  if (dist_bits == 32)
    return a.g.adjp ? launch_d<uint32_t, true, ALGO>(a, team, grid, st)
                    : launch_d<uint32_t, false, ALGO>(a, team, grid, st);
  if (a.g.adjp) return cudaErrorInvalidValue;
  return launch_d<uint64_t, false, ALGO>(a, team, grid, st);
}

// Resident CTAs per SM; for 32-bit distances the smaller of the two adjacency forms.
template <int ALGO>
cudaError_t occupancy_algo(int dist_bits, int team, int* blocks_per_sm) {
  if (dist_bits != 32) return occ_d<uint64_t, false, ALGO>(team, blocks_per_sm);
  int a = 0, b = 0;
  cudaError_t e = occ_d<uint32_t, false, ALGO>(team, &a);
  if (e == cudaSuccess) e = occ_d<uint32_t, true, ALGO>(team, &b);
  *blocks_per_sm = a < b ? a : b;
  return e;
}

}  // namespace
}  // namespace bcgpu
