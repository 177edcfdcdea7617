// Graph preparation (once per graph) and small device helpers.
//
// prep: interleave the CSR column and weight arrays into one {col, w} record
// per entry (one 8-byte load per edge in every pass), and compute
// Delta_node(v) = min weight incident to v (Sec. 3.2, before Eq. 2), one warp
// per vertex.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "bc_common.h"

namespace bcgpu {
namespace {

__global__ void pack_adj_kernel(uint64_t nnz, const uint32_t* __restrict__ col, const uint32_t* __restrict__ w,
                                uint2* __restrict__ adj) {
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < nnz; e += (uint64_t)gridDim.x * blockDim.x)
    adj[e] = make_uint2(col[e], w[e]);
}

__global__ void pack32_kernel(uint64_t nnz, const uint32_t* __restrict__ col, const uint32_t* __restrict__ w,
                              uint32_t col_bits, uint32_t* __restrict__ adjp) {
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < nnz; e += (uint64_t)gridDim.x * blockDim.x)
    adjp[e] = col[e] | (w[e] << col_bits);
}

// One warp per row: the smallest weight (Delta_node), and optionally the
// second smallest (counting repeats) and the neighbour of the smallest (the
// lowest id among equal weights).
__global__ void dnode_kernel(uint32_t n, const uint64_t* __restrict__ row_ptr, const uint32_t* __restrict__ col,
                             const uint32_t* __restrict__ w, uint32_t* __restrict__ dnode,
                             uint32_t* __restrict__ dnode2, uint32_t* __restrict__ dnode_arg) {
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  for (uint64_t v = warp; v < n; v += nwarps) {
    uint32_t m1 = 0xffffffffu, m2 = 0xffffffffu, a1 = 0xffffffffu;
    for (uint64_t e = row_ptr[v] + lane; e < row_ptr[v + 1]; e += 32) {
      const uint32_t x = w[e];
      const uint32_t c = col[e];
      if (x < m1 || (x == m1 && c < a1)) {
        m2 = m1;
        m1 = x;
        a1 = c;
      } else if (x < m2) {
        m2 = x;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const uint32_t o1 = __shfl_xor_sync(0xffffffffu, m1, o);
      const uint32_t o2 = __shfl_xor_sync(0xffffffffu, m2, o);
      const uint32_t oa = __shfl_xor_sync(0xffffffffu, a1, o);
      // the two smallest of both lanes' pairs; the smaller first weight keeps its neighbour
      const uint32_t n2 = min(min(m2, o2), max(m1, o1));
      if (o1 < m1 || (o1 == m1 && oa < a1)) {
        m1 = o1;
        a1 = oa;
      }
      m2 = n2;
    }
    if (lane == 0) {
      dnode[v] = m1;
      if (dnode2) dnode2[v] = m2;
      if (dnode_arg) dnode_arg[v] = a1;
    }
  }
}

__global__ void fill_u64_kernel(uint64_t* p, uint64_t count, uint64_t value) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x)
    p[i] = value;
}

__global__ void scale_kernel(double* p, uint64_t count, double s) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x)
    p[i] *= s;
}

__global__ void check_sources_kernel(const uint32_t* src, uint32_t k, uint32_t n, int* err) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x)
    if (src[i] >= n) atomicCAS(err, DEV_OK, DEV_ERR_INVALID);
}

__global__ void fill_slabs_kernel(char* base, uint64_t stride, uint32_t nslots, uint64_t off, uint64_t words,
                                  uint32_t value) {
  for (uint32_t slot = blockIdx.y; slot < nslots; slot += gridDim.y) {
    uint32_t* p = reinterpret_cast<uint32_t*>(base + (uint64_t)slot * stride + off);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < words; i += (uint64_t)gridDim.x * blockDim.x)
      p[i] = value;
  }
}

int grid_for(uint64_t work, int block) {
  uint64_t g = (work + block - 1) / block;
  if (g < 1) g = 1;
  if (g > 152ull * 32) g = 152ull * 32;
  return (int)g;
}

}  // namespace

cudaError_t launch_prep(uint32_t n, uint64_t nnz, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* w,
                        uint2* adj, uint32_t* dnode, uint32_t* dnode2, uint32_t* dnode_arg, cudaStream_t st) {
  if (nnz > 0 && adj) pack_adj_kernel<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, col, w, adj);
  dnode_kernel<<<grid_for((uint64_t)n * 32, 256), 256, 0, st>>>(n, row_ptr, col, w, dnode, dnode2, dnode_arg);
  return cudaGetLastError();
}

cudaError_t launch_pack32(uint64_t nnz, const uint32_t* col, const uint32_t* w, uint32_t col_bits, uint32_t* adjp,
                          cudaStream_t st) {
  if (nnz == 0) return cudaSuccess;
  pack32_kernel<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, col, w, col_bits, adjp);
  return cudaGetLastError();
}

cudaError_t launch_fill_u64(uint64_t* p, uint64_t count, uint64_t value, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  fill_u64_kernel<<<grid_for(count, 256), 256, 0, st>>>(p, count, value);
  return cudaGetLastError();
}

cudaError_t launch_scale(double* p, uint64_t count, double scale, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  scale_kernel<<<grid_for(count, 256), 256, 0, st>>>(p, count, scale);
  return cudaGetLastError();
}

cudaError_t launch_check_sources(const uint32_t* src, uint32_t k, uint32_t n, int* err, cudaStream_t st) {
  if (k == 0) return cudaSuccess;
  check_sources_kernel<<<grid_for(k, 256), 256, 0, st>>>(src, k, n, err);
  return cudaGetLastError();
}

cudaError_t launch_fill_slabs(char* base, uint64_t stride, uint32_t nslots, uint64_t off, uint64_t bytes,
                              uint32_t value, cudaStream_t st) {
  if (nslots == 0 || bytes == 0) return cudaSuccess;
  const uint64_t words = bytes / 4;
  dim3 grid((unsigned)std::min<uint64_t>((words + 255) / 256, 64), std::min<uint32_t>(nslots, 65535));
  fill_slabs_kernel<<<grid, 256, 0, st>>>(base, stride, nslots, off, words, value);
  return cudaGetLastError();
}

}  // namespace bcgpu
