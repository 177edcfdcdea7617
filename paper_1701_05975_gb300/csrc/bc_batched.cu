// Strict schedule instantiations of the batched kernel (device code in
// bc_batched.cuh) and the launch entry points used by the API layer.
#include "bc_batched.cuh"

namespace bcgpu {

int batched_block_threads(int team) { return team == 32 ? 256 : team; }

cudaError_t launch_batched(const BatchArgs& a, int dist_bits, int team, int grid, cudaStream_t st) {
  if (a.algo == ALGO_DELTA) return launch_batched_delta(a, dist_bits, team, grid, st);
  return launch_algo<ALGO_STRICT>(a, dist_bits, team, grid, st);
}

cudaError_t batched_occupancy(int dist_bits, int team, int algo, int* blocks_per_sm) {
  if (algo == ALGO_DELTA) return batched_occupancy_delta(dist_bits, team, blocks_per_sm);
  return occupancy_algo<ALGO_STRICT>(dist_bits, team, blocks_per_sm);
}

cudaError_t batched_occupancy(int dist_bits, int team, int* blocks_per_sm) {
  return batched_occupancy(dist_bits, team, ALGO_STRICT, blocks_per_sm);
}

}  // namespace bcgpu
