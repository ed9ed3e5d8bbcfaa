// Persistent ensemble kernel, FP32 instantiation (ps_persist.cuh).
#include "ps_persist.cuh"

namespace ps {
cudaError_t ens_launch_f32(const EnsLaunch& L, int grid, size_t smem, cudaStream_t s) {
  return ens_launch_t<float>(L, grid, smem, s);
}
cudaError_t ens_blocks_per_sm_f32(size_t smem, int* per_sm) { return ens_blocks_per_sm_t<float>(smem, per_sm); }
}  // namespace ps
