// Batched ensemble passes, float instantiation (ps_batch.cuh).
#include "ps_batch.cuh"

namespace ps {

cudaError_t batch_pass_f32(int kind, int n, const BatchArgs& b, const Geo& g, int M, cudaStream_t s) {
  switch (n) {
    case 32: return batch_pass_n<float, 32>(kind, b, g, M, s);
    case 48: return batch_pass_n<float, 48>(kind, b, g, M, s);
    case 64: return batch_pass_n<float, 64>(kind, b, g, M, s);
    case 96: return batch_pass_n<float, 96>(kind, b, g, M, s);
    case 128: return batch_pass_n<float, 128>(kind, b, g, M, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t batch_update_f32(const BatchArgs& b, const Geo& g, int M, int full, cudaStream_t s) {
  return batch_update<float>(b, g, M, full, s);
}

// Energy of the step statistics of member blockIdx.x: sum of its z-inverse
// partials (n of them) into its stats word (same order as k_sum_partials).
__global__ void __launch_bounds__(256) k_batch_sum(const __grid_constant__ BatchArgs B, const int n, double* const* out) {
  __shared__ double red[32];
  const PassArgs& a = B.args[blockIdx.x];
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += a.e_part[i];
  const double t = block_sum(v, red);
  if (threadIdx.x == 0) *out[blockIdx.x] = t;
}

cudaError_t batch_sum(const BatchArgs& b, int n, double* const* out, int M, cudaStream_t s) {
  k_batch_sum<<<M, 256, 0, s>>>(b, n, out);
  return cudaGetLastError();
}

}  // namespace ps
