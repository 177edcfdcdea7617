// Delta-stepping schedule instantiations of the batched kernel (device code
// in bc_batched.cuh).
#include "bc_batched.cuh"

namespace bcgpu {

cudaError_t launch_batched_delta(const BatchArgs& a, int dist_bits, int team, int grid, cudaStream_t st) {
  return launch_algo<ALGO_DELTA>(a, dist_bits, team, grid, st);
}

cudaError_t batched_occupancy_delta(int dist_bits, int team, int* blocks_per_sm) {
  return occupancy_algo<ALGO_DELTA>(dist_bits, team, blocks_per_sm);
}

}  // namespace bcgpu
