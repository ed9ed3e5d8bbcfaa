// zinv pass, float instantiations for every supported line length.
#include "ps_passes.cuh"

namespace ps {

template <>
cudaError_t launch_zinv<float>(const PassArgs& a, cudaStream_t s, int* nb) {
#define CALL(N) zinv_n<float, N>(a, s, nb)
  PS_DISPATCH_N(a.g.nz, CALL)
#undef CALL
}

template <int N>
static int zinv_blocks_n(const Geo& g, int var) {
  const int b0 = zinv_grid_blocks<float, N, 0>(g);
  if constexpr (HasShapes<float, N>::v) {
    const int b1 = zinv_grid_blocks<float, N, 1>(g), b2 = zinv_grid_blocks<float, N, 2>(g);
    if (var < 0) return b0 > b1 ? (b0 > b2 ? b0 : b2) : (b1 > b2 ? b1 : b2);
    if (var == 1) return b1;
    if (var == 2 && AltE<float, N>::v != EOf<float, N>::v) return b2;
  }
  return b0;
}

template <>
int zinv_blocks<float>(const Geo& g, int var) {
#define CALL(N) zinv_blocks_n<N>(g, var)
  switch (g.nz) {
    case 8: return CALL(8);
    case 16: return CALL(16);
    case 32: return CALL(32);
    case 48: return CALL(48);
    case 64: return CALL(64);
    case 96: return CALL(96);
    case 128: return CALL(128);
    case 192: return CALL(192);
    case 256: return CALL(256);
    case 512: return CALL(512);
    case 1024: return CALL(1024);
    default: return 0;
  }
#undef CALL
}

template <int N>
static bool pass_shape_n(int k, int var, int* cols, int* points) {
  if (var != 0 && !HasShapes<float, N>::v) return false;
  if (var == 2 && AltE<float, N>::v == EOf<float, N>::v) return false;
  if (var < 0 || var > 2 || k < 0 || k > 2) return false;
  auto put = [&](int tx, int e) {
    *cols = tx;
    *points = e;
    return true;
  };
#define SHP(K, V) put(ColShape<float, N, K, V>::TX, ColShape<float, N, K, V>::E)
  if constexpr (HasShapes<float, N>::v) {
    if (var == 1) return k == 0 ? SHP(0, 1) : k == 1 ? SHP(1, 1) : SHP(2, 1);
    if (var == 2) return k == 0 ? SHP(0, 2) : k == 1 ? SHP(1, 2) : SHP(2, 2);
  }
  return k == 0 ? SHP(0, 0) : k == 1 ? SHP(1, 0) : SHP(2, 0);
#undef SHP
}

template <>
bool pass_shape<float>(int k, int n, int var, int* cols, int* points) {
  switch (n) {
    case 8: return pass_shape_n<8>(k, var, cols, points);
    case 16: return pass_shape_n<16>(k, var, cols, points);
    case 32: return pass_shape_n<32>(k, var, cols, points);
    case 48: return pass_shape_n<48>(k, var, cols, points);
    case 64: return pass_shape_n<64>(k, var, cols, points);
    case 96: return pass_shape_n<96>(k, var, cols, points);
    case 128: return pass_shape_n<128>(k, var, cols, points);
    case 192: return pass_shape_n<192>(k, var, cols, points);
    case 256: return pass_shape_n<256>(k, var, cols, points);
    case 512: return pass_shape_n<512>(k, var, cols, points);
    case 1024: return pass_shape_n<1024>(k, var, cols, points);
    default: return false;
  }
}

}  // namespace ps
