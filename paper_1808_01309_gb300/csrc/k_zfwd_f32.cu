// zfwd pass, float instantiations for every supported line length.
#include "ps_passes.cuh"

namespace ps {

template <>
cudaError_t launch_zfwd<float>(const PassArgs& a, cudaStream_t s) {
#define CALL(N) zfwd_n<float, N>(a, s)
  PS_DISPATCH_N(a.g.nz, CALL)
#undef CALL
}

template <>
cudaError_t launch_update<float>(const PassArgs& a, cudaStream_t s) {
  return update_launch<float>(a, s);
}

}  // namespace ps
