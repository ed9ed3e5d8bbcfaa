// yfwd pass, float instantiations for every supported line length.
#include "ps_passes.cuh"

namespace ps {

template <>
cudaError_t launch_yfwd<float>(const PassArgs& a, cudaStream_t s) {
#define CALL(N) yfwd_n<float, N>(a, s)
  PS_DISPATCH_N(a.g.ny, CALL)
#undef CALL
}

}  // namespace ps
