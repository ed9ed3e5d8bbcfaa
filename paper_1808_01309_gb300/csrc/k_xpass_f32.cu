// xpass pass, float instantiations for every supported line length.
#include "ps_passes.cuh"

namespace ps {

template <>
cudaError_t launch_xpass<float>(const PassArgs& a, cudaStream_t s) {
#define CALL(N) xpass_n<float, N>(a, s)
  PS_DISPATCH_N(a.g.nx, CALL)
#undef CALL
}

}  // namespace ps
