// zinv pass, double instantiations for every supported line length.
#include "ps_passes.cuh"

namespace ps {

template <>
cudaError_t launch_zinv<double>(const PassArgs& a, cudaStream_t s, int* nb) {
#define CALL(N) zinv_n<double, N>(a, s, nb)
  PS_DISPATCH_N(a.g.nz, CALL)
#undef CALL
}

template <>
int zinv_blocks<double>(const Geo& g) {
  int nb = 0;
  switch (g.nz) {
#define CASE(N) case N: nb = NBOf<double, N>::v; break;
    CASE(8) CASE(16) CASE(32) CASE(48) CASE(64) CASE(96) CASE(128) CASE(192) CASE(256) CASE(512) CASE(1024)
#undef CASE
    default: return 0;
  }
  return (g.kxp / TXOf<double>::v) * ((g.cy + nb - 1) / nb);
}

}  // namespace ps
