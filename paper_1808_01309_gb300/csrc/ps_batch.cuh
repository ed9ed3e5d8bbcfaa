// Batched ensemble passes: members of one grid size (same nx, ny, nz,
// precision and dealiasing; their own states, viscosities and forcing)
// share one launch per pass.  Each launch covers the CTA tiles of every
// member (blockIdx.y = member for the column passes and the update; the x
// pass keeps its persistent TMA-staged loop, over the (member, row group)
// pairs), and each pass kind keeps the register and shared-memory budget of
// its own kernel.  The tile functions are those of the per-pass kernels
// (ps_passes.cuh), reading each member's arguments from a device array.
#pragma once
#include "ps_passes.cuh"

namespace ps {

// Up to BATCH_MAX members per launch, their arguments in the kernel's
// parameter space (constant bank: broadcast reads, never reloaded after the
// passes' stores, as for the per-pass kernels); larger classes take several
// launches.  32 x about 430 bytes stays well inside the 32 KB parameter limit.
constexpr int BATCH_MAX = 32;
struct BatchArgs {
  PassArgs args[BATCH_MAX];  // one per member
  int gx, gy;                // column passes: tile grid of one member (z: fields)
  int full;                  // update: caller layout
};
static_assert(sizeof(BatchArgs) < 32000, "kernel parameter space");

template <typename T, int N>
__global__ void __launch_bounds__(ColShape<T, N, 0>::NTH, MinB<T, N>::zinv) k_batch_zinv(const __grid_constant__ BatchArgs B) {
  const PassArgs& a = B.args[blockIdx.y];
  // the step statistics start from zero (the x pass of this stage takes the maximum)
  if (a.umax2 && blockIdx.x == 0 && threadIdx.x == 0) *a.umax2 = 0ull;
  const int t = blockIdx.x;
  zinv_tile<T, N, 1, 0, false, 0>(a, WorkTile{t % B.gx, t / B.gx, 0, B.gx});
}

template <typename T, int N, int K>  // K: 0 y-inverse, 1 y-forward, 2 z-forward
__global__ void __launch_bounds__(ColShape<T, N, K == 2 ? 2 : 1>::NTH, K == 2 ? MinB<T, N>::zfwd : MinB<T, N>::ypass)
    k_batch_col(const __grid_constant__ BatchArgs B) {
  const PassArgs& a = B.args[blockIdx.y];
  const int t = blockIdx.x, gxy = B.gx * B.gy;
  const WorkTile tl{(t % gxy) % B.gx, (t % gxy) / B.gx, t / gxy, B.gx};
  if constexpr (K == 0) yinv_tile<T, N, false, 0>(a, tl);
  else if constexpr (K == 1) yfwd_tile<T, N, false, 0>(a, tl);
  else zfwd_tile<T, N, false, 0>(a, tl);
}

template <typename T>
__global__ void __launch_bounds__(256) k_batch_update(const __grid_constant__ BatchArgs B) {
  update_mode<T, 1, 0, false, false>(B.args[blockIdx.y], B.full, blockIdx.x * blockDim.x + threadIdx.x);
}

// x pass over the row groups of M members: CTAs loop over the pairs
// (member, group) = (it / ng, it % ng) with the TMA stage of k_xpass.
template <typename T, int N>
__global__ void __launch_bounds__(RPCOf<T, N>::v * (N / EPass<T, N, 3>::v), MinB<T, N>::xpass)
    k_batch_xpass(const __grid_constant__ BatchArgs B, const int M, const int rpc) {
  using V = typename cplx<T>::type;
  constexpr int E = EPass<T, N, 3>::v, G = N / E;
  constexpr int NF = 6;
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ double red[32];
  __shared__ __align__(8) uint64_t bar[1];
  __shared__ int abort_flag;
  const Geo& g = B.args[0].g;  // every member has this geometry
  const int kxp = g.kxp;
  const int tid = threadIdx.x;
  const int j0 = tid % G, rl = tid / G;
  const long long rows = (long long)g.nz * g.ny;
  const long long ng = (rows + rpc - 1) / rpc;
  const long long total = ng * M;
  V* stage = reinterpret_cast<V*>(smraw);
  V* exbuf = stage + NF * rpc * kxp;
  LinesExchange<V, 1> ex{exbuf + rl * XLINES * N, N, 0, 0};
  if (G >= 32) {
    ex.bar_id = 1 + rl;
    ex.nthr = G;
  } else {
    ex.bar_id = -1;
  }
  // every member has the same twiddles (same nx): those of member 0
  constexpr bool TR = XTwReg<T, N>::v;
  constexpr bool TT = !TR && XTwTable<T, N>::v;
  using TwAcc = typename std::conditional<TR, RegTw<V, N, E>,
                typename std::conditional<TT, ThreadTw<V, N, E>, GlobalTw<V>>::type>::type;
  TwAcc tw;
  if constexpr (TR) {
    tw.load(static_cast<const V*>(B.args[0].tw_x), j0);
  } else if constexpr (TT) {
    V* twt = exbuf + rpc * XLINES * N;
    if (rl == 0) fill_thread_tw<N, E>(twt, static_cast<const V*>(B.args[0].tw_x), j0);
    tw = TwAcc{twt, j0};
  } else {
    tw = TwAcc{static_cast<const V*>(B.args[0].tw_x)};
  }
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    abort_flag = 0;
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](long long pair) {
    const int m = (int)(pair / ng);
    const long long r0 = (pair - (long long)m * ng) * rpc;
    const long long nr = rows - r0 < rpc ? rows - r0 : rpc;
    const uint32_t bytes = (uint32_t)(nr * kxp * sizeof(V));
    const V* src = static_cast<const V*>(B.args[m].b6);
    mbar_arrive_expect_tx(&bar[0], (uint32_t)NF * bytes);
    for (int c = 0; c < NF; ++c) bulk_g2s(stage + c * rpc * kxp, src + ((long long)c * rows + r0) * kxp, bytes, &bar[0]);
  };
  uint32_t ph = 0u;
  long long it = blockIdx.x;
  bool inflight = false;
  if (tid == 0 && it < total) {
    issue(it);
    inflight = true;
  }
  T umax2 = 0;
  int mcur = it < total ? (int)(it / ng) : 0;
  while (it < total) {
    const long long nxt = it + gridDim.x;
    const int m = (int)(it / ng);
    if (m != mcur) {  // the maximum of the previous member is complete for this CTA
      if (B.args[mcur].umax2) {
        const double t = block_max((double)umax2, red);
        if (tid == 0) atomicMax(B.args[mcur].umax2, (unsigned long long)__double_as_longlong(t));
      }
      umax2 = 0;
      mcur = m;
    }
    const uint32_t cur = ph;
    ph ^= 1u;
    if (!mbar_wait(&bar[0], cur, PS_WAIT_LIMIT)) abort_flag = 1;
    __syncthreads();
    if (abort_flag) {
      if (tid == 0) {
        atomicExch(B.args[m].err, PS_DEV_TIMEOUT_XPASS);
        if (inflight) mbar_wait(&bar[0], cur, PS_DRAIN_LIMIT);
      }
      break;
    }
    const PassArgs& a = B.args[m];
    const long long row = (it - (long long)m * ng) * rpc + rl;
    xpass_row<T, N, 1, 0, false>(a, row, row < rows, j0, stage + rl * kxp, (long long)rpc * kxp, tw, ex, umax2, [&] {
      __syncthreads();
      if (tid == 0) {
        inflight = nxt < total;
        if (inflight) {
          fence_proxy_async();
          issue(nxt);
        }
      }
    });
    __syncthreads();
    it = nxt;
  }
  if (B.args[mcur].umax2 && !abort_flag) {
    const double t = block_max((double)umax2, red);
    if (tid == 0) atomicMax(B.args[mcur].umax2, (unsigned long long)__double_as_longlong(t));
  }
}

// ---- launchers (grid shapes as the per-pass launchers) -------------------

template <typename T, int N>
cudaError_t batch_zinv(const BatchArgs& b0, const Geo& g, int M, cudaStream_t s) {
  using V = typename cplx<T>::type;
  using SH = ColShape<T, N, 0>;
  BatchArgs b = b0;
  b.gx = g.kxp / SH::TX;
  b.gy = (g.cy + SH::NB - 1) / SH::NB;
  const size_t smem = (1ull * SH::NB * N * SH::TX + 3ull * SH::NB * g.cz * SH::TX) * sizeof(V);
  cudaError_t e = prep(k_batch_zinv<T, N>, smem);
  if (e != cudaSuccess) return e;
  k_batch_zinv<T, N><<<dim3(b.gx * b.gy, M), SH::NTH, smem, s>>>(b);
  return cudaGetLastError();
}

template <typename T, int N, int K>
cudaError_t batch_col(const BatchArgs& b0, const Geo& g, int M, int nf, cudaStream_t s) {
  using V = typename cplx<T>::type;
  using SH = ColShape<T, N, K == 2 ? 2 : 1>;
  BatchArgs b = b0;
  b.gx = g.kxp / SH::TX;
  b.gy = K == 2 ? (g.cy + SH::NB - 1) / SH::NB : (g.nz + SH::NB - 1) / SH::NB;
  const size_t smem = (size_t)ColBuf<T, N>::v * SH::NB * N * SH::TX * sizeof(V);
  cudaError_t e = prep(k_batch_col<T, N, K>, smem);
  if (e != cudaSuccess) return e;
  k_batch_col<T, N, K><<<dim3(b.gx * b.gy * nf, M), SH::NTH, smem, s>>>(b);
  return cudaGetLastError();
}

template <typename T, int N>
cudaError_t batch_xpass(const BatchArgs& b, const Geo& g, int M, cudaStream_t s) {
  constexpr int G = N / EPass<T, N, 3>::v;
  int rpc = RPCOf<T, N>::v;
  while (rpc > 1 && xpass_smem<T, N>(g, rpc, 6) > 113 * 1024) rpc /= 2;
  const size_t smem = xpass_smem<T, N>(g, rpc, 6);
  cudaError_t e = cudaFuncSetAttribute(k_batch_xpass<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_xpass<T, N>, rpc * G, smem)) != cudaSuccess)
    return e;
  const long long rows = (long long)g.nz * g.ny;
  const long long pairs = (rows + rpc - 1) / rpc * M;
  long long grid = (long long)nsm * (per_sm > 0 ? per_sm : 1);
  if (grid > pairs) grid = pairs;
  k_batch_xpass<T, N><<<(unsigned)grid, rpc * G, smem, s>>>(b, M, rpc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t batch_update(const BatchArgs& b0, const Geo& g, int M, int full, cudaStream_t s) {
  BatchArgs b = b0;
  b.full = full;
  const long long n = full ? (long long)g.nz * g.ny * g.nh : (long long)g.cz * g.cy * g.cx;
  if (n >= (1LL << 32) - 256) return cudaErrorInvalidValue;
  k_batch_update<T><<<dim3((unsigned)((n + 255) / 256), M), 256, 0, s>>>(b);
  return cudaGetLastError();
}

// One pass of kind `kind` (0 z-inverse, 1 y-inverse, 2 x, 3 y-forward,
// 4 z-forward) for M members of geometry g, lines of n points.
template <typename T, int N>
cudaError_t batch_pass_n(int kind, const BatchArgs& b, const Geo& g, int M, cudaStream_t s) {
  switch (kind) {
    case 0: return batch_zinv<T, N>(b, g, M, s);
    case 1: return batch_col<T, N, 0>(b, g, M, 6, s);
    case 2: return batch_xpass<T, N>(b, g, M, s);
    case 3: return batch_col<T, N, 1>(b, g, M, 3, s);
    case 4: return batch_col<T, N, 2>(b, g, M, 3, s);
    default: return cudaErrorInvalidValue;
  }
}

// Launchers for FP32 and FP64 (ps_batch_f32.cu, ps_batch_f64.cu): pass
// `kind` on lines of n points; cudaErrorInvalidValue for lengths outside
// {32, 48, 64, 96, 128}.
cudaError_t batch_pass_f32(int kind, int n, const BatchArgs& b, const Geo& g, int M, cudaStream_t s);
cudaError_t batch_pass_f64(int kind, int n, const BatchArgs& b, const Geo& g, int M, cudaStream_t s);
cudaError_t batch_update_f32(const BatchArgs& b, const Geo& g, int M, int full, cudaStream_t s);
cudaError_t batch_update_f64(const BatchArgs& b, const Geo& g, int M, int full, cudaStream_t s);
cudaError_t batch_sum(const BatchArgs& b, int n, double* const* out, int M, cudaStream_t s);

}  // namespace ps
