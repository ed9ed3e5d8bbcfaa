// Batched ensemble passes, double instantiation (ps_batch.cuh).
#include "ps_batch.cuh"

namespace ps {

cudaError_t batch_pass_f64(int kind, int n, const BatchArgs& b, const Geo& g, int M, cudaStream_t s) {
  switch (n) {
    case 32: return batch_pass_n<double, 32>(kind, b, g, M, s);
    case 48: return batch_pass_n<double, 48>(kind, b, g, M, s);
    case 64: return batch_pass_n<double, 64>(kind, b, g, M, s);
    case 96: return batch_pass_n<double, 96>(kind, b, g, M, s);
    case 128: return batch_pass_n<double, 128>(kind, b, g, M, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t batch_update_f64(const BatchArgs& b, const Geo& g, int M, int full, cudaStream_t s) {
  return batch_update<double>(b, g, M, full, s);
}

}  // namespace ps
