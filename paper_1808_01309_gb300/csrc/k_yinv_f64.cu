// yinv pass, double instantiations for every supported line length.
#include "ps_passes.cuh"

namespace ps {

template <>
cudaError_t launch_yinv<double>(const PassArgs& a, cudaStream_t s) {
#define CALL(N) yinv_n<double, N>(a, s)
  PS_DISPATCH_N(a.g.ny, CALL)
#undef CALL
}

}  // namespace ps
