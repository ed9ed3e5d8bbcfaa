// Persistent ensemble kernel, FP64 instantiation (ps_persist.cuh).
#include "ps_persist.cuh"

namespace ps {
cudaError_t ens_launch_f64(const EnsLaunch& L, int grid, size_t smem, cudaStream_t s) {
  return ens_launch_t<double>(L, grid, smem, s);
}
cudaError_t ens_blocks_per_sm_f64(size_t smem, int* per_sm) { return ens_blocks_per_sm_t<double>(smem, per_sm); }
}  // namespace ps
