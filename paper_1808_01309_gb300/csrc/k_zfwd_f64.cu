// zfwd pass, double instantiations for every supported line length.
#include "ps_passes.cuh"

namespace ps {

template <>
cudaError_t launch_zfwd<double>(const PassArgs& a, cudaStream_t s) {
#define CALL(N) zfwd_n<double, N>(a, s)
  PS_DISPATCH_N(a.g.nz, CALL)
#undef CALL
}

template <>
cudaError_t launch_update<double>(const PassArgs& a, cudaStream_t s) {
  return update_launch<double>(a, s);
}

}  // namespace ps
