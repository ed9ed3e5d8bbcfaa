// Persistent ensemble launch: every pass of every RK stage of every member of
// an ensemble of independent solves, for several steps, in ONE kernel launch.
//
// Work queue.  The host lists the pass instances (member, step, stage, pass)
// in a topological order: for each step and stage, all members' z-inverse
// passes, then all members' y-inverse passes, and so on.  Pass instance i owns
// the tickets [tick0_i, tick0_i + ceil(ntiles_i / per_i)); a ticket stands for
// `per` consecutive tiles (the CTA tiles of the per-pass kernels).  CTAs take
// tickets in increasing order from one device counter.  Before the first
// ticket of a pass instance a CTA waits until every tile of the member's
// previous pass instance is done (done[dep] == need: release/acquire through
// one counter per pass instance); after its tiles it adds their count to the
// pass instance's counter.  A CTA only waits for lower tickets, which CTAs
// already running hold, so the queue always advances however many CTAs are
// resident.  Every wait is bounded: when it runs out, or another CTA has
// already reported a failure, the CTA writes the error word and leaves.
//
// Within one launch a pass reads what other CTAs wrote earlier in the same
// launch, so the tile functions are instantiated with COH = true: their data
// loads are ordinary coherent loads (not the read-only path), which the
// acquire of the previous pass's counter orders after that pass's writes (the
// acquire also orders the z-inverse tile's cp.async staging).  Twiddles and
// integrating-factor tables are written before the launch and keep the
// read-only path.
//
// Supported members: FP32 or FP64, the hydrodynamic system without a learned
// closure, each axis in {32, 48, 64, 96, 128} (every pass then has 256
// threads per tile, the CTA size of this kernel).
#pragma once
#include "ps_passes.cuh"

namespace ps {

enum EnsKind : int { EK_ZINV = 0, EK_YINV = 1, EK_XPASS = 2, EK_YFWD = 3, EK_ZFWD = 4, EK_UPDATE = 5, EK_SUM = 6 };
constexpr int ENS_THREADS = 256;
constexpr int ENS_UPDATE_MODES = 256;  // modes per update tile (one per thread)
constexpr int PS_DEV_TIMEOUT_ENSEMBLE = 3;

// One pass instance of the persistent launch.
struct EnsPass {
  long long tick0;     // first ticket
  int args;            // index into the launch's PassArgs
  int kind;            // EnsKind
  int n;               // line length of the pass axis (column and x passes)
  int ntiles;          // tiles of the pass instance
  int per;             // tiles per ticket
  int gx, gy;          // tile grid along x and y (column passes); SUM: partial count
  int dep;             // pass instance that must be complete first, or -1
  int need;            // its tile count
  int full;            // update: the caller's layout (last RK stage)
  double* sum_out;     // SUM: destination of the energy sum
};

struct EnsLaunch {
  const EnsPass* passes;
  int npass;
  const PassArgs* args;
  unsigned* done;            // completed tiles per pass instance (zero at launch)
  unsigned long long* head;  // next ticket (zero at launch)
  long long tickets;         // total tickets
  int* err;                  // error word (zero at launch)
  unsigned polls;            // polls before a dependency wait gives up
};

// Tile grid and dynamic shared memory of one pass kind for geometry g.
struct EnsShape {
  int ntiles = 0, gx = 0, gy = 0;
  size_t smem = 0;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_i32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// x pass on the ENS_THREADS / G consecutive rows of tile `tile`, reading its
// input rows from global memory (written by the y-inverse pass of this launch).
// FP32 128-point rows take 8 points per thread here (three stages): with 16
// (two stages) this tile alone made the whole kernel spill at its 128
// registers.
template <typename T, int N> struct EnsXE {
  static constexpr int v = sizeof(T) == 4 && N == 128 ? 8 : EPass<T, N, 3>::v;
};
template <typename T, int N>
__device__ __forceinline__ void ens_xpass_tile(const PassArgs& a, const int tile) {
  using V = typename cplx<T>::type;
  constexpr int E = EnsXE<T, N>::v, G = N / E, RPC = ENS_THREADS / G;
  static_assert(G < 32, "rows of one tile share warps (warp-synchronous exchanges)");
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ double red[32];
  const int tid = threadIdx.x, j0 = tid % G, rl = tid / G;
  LinesExchange<V, 1> ex{reinterpret_cast<V*>(smraw) + rl * XLINES * N, N, 0, 0};
  ex.bar_id = -1;
  const GlobalTw<V> tw{static_cast<const V*>(a.tw_x)};
  const long long rows = (long long)a.g.nz * a.g.ny;
  const long long row = (long long)tile * RPC + rl;
  const bool rvalid = row < rows;
  const V* B = static_cast<const V*>(a.b6) + (rvalid ? row : 0) * a.g.kxp;
  T umax2 = 0;
  auto none = [] {};
  xpass_row<T, N, 1, 0, true, GlobalTw<V>, decltype(none)&, E>(a, row, rvalid, j0, B, rows * a.g.kxp, tw, ex, umax2,
                                                                none);
  if (a.umax2) {
    const double t = block_max((double)umax2, red);
    if (tid == 0) atomicMax(a.umax2, (unsigned long long)__double_as_longlong(t));
  }
}

template <typename T, int N>
__device__ __forceinline__ void ens_tile_n(const EnsPass& P, const PassArgs& a, const int tile) {
  static_assert(ColThreads<T, N, 0>::v == ENS_THREADS && ColThreads<T, N, 1>::v == ENS_THREADS &&
                    ColThreads<T, N, 2>::v == ENS_THREADS,
                "column tiles of ENS_THREADS threads");
  const int gx = P.gx, gxy = P.gx * P.gy;
  const WorkTile tl{(tile % gxy) % gx, (tile % gxy) / gx, tile / gxy, gx};
  switch (P.kind) {
    case EK_ZINV: zinv_tile<T, N, 1, 0, true, 0>(a, tl); break;
    case EK_YINV: yinv_tile<T, N, true, 0>(a, tl); break;
    case EK_XPASS: ens_xpass_tile<T, N>(a, tile); break;
    case EK_YFWD: yfwd_tile<T, N, true, 0>(a, tl); break;
    case EK_ZFWD: zfwd_tile<T, N, true, 0>(a, tl); break;
    default: break;
  }
}

template <typename T>
__device__ __forceinline__ void ens_tile(const EnsPass& P, const PassArgs& a, const int tile) {
  if (P.kind == EK_UPDATE) {
    update_mode<T, 1, 0, false, true>(a, P.full, (unsigned)tile * ENS_UPDATE_MODES + threadIdx.x);
    return;
  }
  if (P.kind == EK_SUM) {
    __shared__ double red[32];
    double v = 0.0;
    for (int i = threadIdx.x; i < P.gx; i += blockDim.x) v += a.e_part[i];
    const double t = block_sum(v, red);
    if (threadIdx.x == 0) *P.sum_out = t;
    return;
  }
  switch (P.n) {
    case 32: ens_tile_n<T, 32>(P, a, tile); break;
    case 48: ens_tile_n<T, 48>(P, a, tile); break;
    case 64: ens_tile_n<T, 64>(P, a, tile); break;
    case 96: ens_tile_n<T, 96>(P, a, tile); break;
    case 128: ens_tile_n<T, 128>(P, a, tile); break;
    default: break;
  }
}

template <typename T> struct EnsMinB { static constexpr int v = sizeof(T) == 4 ? 2 : 1; };

template <typename T>
__global__ void __launch_bounds__(ENS_THREADS, EnsMinB<T>::v) k_ensemble(const EnsLaunch L) {
  __shared__ long long s_tick;
  __shared__ int s_stop;
  // the current pass instance's arguments (read by every tile: kept in shared
  // memory rather than read from global memory after every store)
  __shared__ __align__(16) PassArgs s_args;
  const int tid = threadIdx.x;
  int cur = 0, ready = -1, loaded = -1;
  for (;;) {
    if (tid == 0) s_tick = (long long)atomicAdd(L.head, 1ull);
    __syncthreads();
    const long long t = s_tick;
    if (t >= L.tickets) break;
    // tickets grow within a CTA: the pass instance cursor only moves forward
    while (cur + 1 < L.npass && L.passes[cur + 1].tick0 <= t) ++cur;
    const EnsPass P = L.passes[cur];  // a register copy (not re-read after the tiles' stores)
    if (cur != ready) {
      if (tid == 0) {
        int stop = 0;
        if (P.dep >= 0) {
          unsigned n = 0;
          while (ld_acquire_u32(L.done + P.dep) < (unsigned)P.need) {
            if (++n >= L.polls || ld_relaxed_i32(L.err) != 0) {
              stop = 1;
              break;
            }
            __nanosleep(100);
          }
          if (stop) atomicCAS(L.err, 0, PS_DEV_TIMEOUT_ENSEMBLE);
        }
        s_stop = stop;
      }
      __syncthreads();
      if (s_stop) break;
      ready = cur;
    }
    if (P.args != loaded) {
      static_assert(sizeof(PassArgs) % 4 == 0, "word copy");
      const int* src = reinterpret_cast<const int*>(L.args + P.args);
      int* dst = reinterpret_cast<int*>(&s_args);
      for (int i = tid; i < (int)(sizeof(PassArgs) / 4); i += blockDim.x) dst[i] = src[i];
      __syncthreads();
      loaded = P.args;
    }
    const PassArgs& a = s_args;
    const int t0 = (int)(t - P.tick0) * P.per;
    const int t1 = t0 + P.per < P.ntiles ? t0 + P.per : P.ntiles;
    for (int tile = t0; tile < t1; ++tile) {
      ens_tile<T>(P, a, tile);
      if (P.kind != EK_UPDATE) __syncthreads();  // the tile's shared memory is reused by the next
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();  // release: the tiles' writes before the count
      atomicAdd(L.done + cur, (unsigned)(t1 - t0));
    }
  }
}

// ---- host side -----------------------------------------------------------

template <typename T, int N>
EnsShape ens_shape_n(int kind, const Geo& g, int nfield) {
  using V = typename cplx<T>::type;
  EnsShape s;
  if (kind == EK_ZINV) {
    constexpr int TX = TXOf<T>::v, NB = NBOf<T, N>::v;
    s.gx = g.kxp / TX;
    s.gy = (g.cy + NB - 1) / NB;
    s.ntiles = s.gx * s.gy;
    s.smem = ((size_t)NB * N * TX + 3ull * NB * g.cz * TX) * sizeof(V);
  } else if (kind == EK_YINV || kind == EK_YFWD) {
    constexpr int TX = TXOf<T, 1>::v, NB = NBOf<T, N, 1>::v;
    s.gx = g.kxp / TX;
    s.gy = (g.nz + NB - 1) / NB;
    s.ntiles = s.gx * s.gy * nfield;
    s.smem = (size_t)ColBuf<T, N>::v * NB * N * TX * sizeof(V);
  } else if (kind == EK_ZFWD) {
    constexpr int TX = TXOf<T, 2>::v, NB = NBOf<T, N, 2>::v;
    s.gx = g.kxp / TX;
    s.gy = (g.cy + NB - 1) / NB;
    s.ntiles = s.gx * s.gy * nfield;
    s.smem = (size_t)ColBuf<T, N>::v * NB * N * TX * sizeof(V);
  } else if (kind == EK_XPASS) {
    constexpr int G = N / EnsXE<T, N>::v, RPC = ENS_THREADS / G;
    const long long rows = (long long)g.nz * g.ny;
    s.ntiles = (int)((rows + RPC - 1) / RPC);
    s.gx = RPC;
    s.smem = (size_t)XLINES * RPC * N * sizeof(V);
  }
  return s;
}

// Shape of pass `kind` on an axis of length n (0 tiles: unsupported length).
template <typename T>
EnsShape ens_shape(int kind, int n, const Geo& g, int nfield) {
  switch (n) {
    case 32: return ens_shape_n<T, 32>(kind, g, nfield);
    case 48: return ens_shape_n<T, 48>(kind, g, nfield);
    case 64: return ens_shape_n<T, 64>(kind, g, nfield);
    case 96: return ens_shape_n<T, 96>(kind, g, nfield);
    case 128: return ens_shape_n<T, 128>(kind, g, nfield);
    default: return EnsShape{};
  }
}

// Launch of the persistent kernel and its resident CTAs per SM for `smem`
// bytes of dynamic shared memory (ps_persist_f32.cu, ps_persist_f64.cu).
cudaError_t ens_launch_f32(const EnsLaunch& L, int grid, size_t smem, cudaStream_t s);
cudaError_t ens_launch_f64(const EnsLaunch& L, int grid, size_t smem, cudaStream_t s);
cudaError_t ens_blocks_per_sm_f32(size_t smem, int* per_sm);
cudaError_t ens_blocks_per_sm_f64(size_t smem, int* per_sm);

template <typename T>
cudaError_t ens_launch_t(const EnsLaunch& L, int grid, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_ensemble<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_ensemble<T><<<grid, ENS_THREADS, smem, s>>>(L);
  return cudaGetLastError();
}

template <typename T>
cudaError_t ens_blocks_per_sm_t(size_t smem, int* per_sm) {
  cudaError_t e = cudaFuncSetAttribute(k_ensemble<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_ensemble<T>, ENS_THREADS, smem);
}

}  // namespace ps
