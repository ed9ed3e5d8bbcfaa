// Learned LES closure on the CUDA path (include/ps.h: ps_plan_set_closure,
// ps_les_training_sample): plain (unpruned) 3D transforms of any number of
// fields, the resolved velocity-gradient invariants, the MLP of ps_mlp.cu, and
// the divergence of the modelled stress that the z-forward pass adds to the
// nonlinear term before the projection.  FP32.
#include <cmath>
#include <string>
#include <vector>

#include "ps.h"
#include "ps_passes.cuh"
#include "ps_tb.cuh"

namespace ps {
void set_last_error(const std::string& msg);

namespace les {

using V = float2;
constexpr int TXG = 8;  // columns per CTA of the strided transform

__global__ void k_tw(V* tw, int n) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  double s, c;
  sincospi(2.0 * m / n, &s, &c);
  tw[m] = make_float2((float)c, (float)(-s));
}

// In-place C2C transform along an axis of length N: element n of line
// (b, col) at (b / nb2) s1 + (b % nb2) s2 + n es + col, col < ncols.
template <int N, int DIR>
__global__ void k_c2c(V* data, const V* __restrict__ tw, int ncols, int nb2, long long s1, long long s2,
                      long long es, int nbatch) {
  constexpr int E = EOf<float, N>::v, G = N / E;
  constexpr int NBG = 256 / (TXG * G) > 0 ? 256 / (TXG * G) : 1;
  extern __shared__ __align__(128) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int tid = threadIdx.x;
  const int line = tid % TXG, rest = tid / TXG, j0 = rest % G, bb = rest / G;
  const int b = blockIdx.y * NBG + bb;
  const int col = blockIdx.x * TXG + line;
  const bool ok = b < nbatch && col < ncols;
  ColumnExchange<V, ilog2<Sched<N, E>::R0>::v> ex{sm + bb * N * TXG, NBG * N * TXG, TXG, line, 0};
  V* base = data + (ok ? (long long)(b / nb2) * s1 + (long long)(b % nb2) * s2 + col : 0);
  V x[E];
#pragma unroll
  for (int m = 0; m < E; ++m) x[m] = ok ? base[(long long)(j0 + m * (N / E)) * es] : czero<V>();
  line_fft<N, E, DIR>(x, j0, tw, ex);
  if (ok) {
#pragma unroll
    for (int m = 0; m < E; ++m) base[(long long)(j0 + m * (N / E)) * es] = x[m];
  }
}

// x rows: spectra of fields 2p and 2p+1 (nh = N/2+1 entries each) <-> real
// rows of N points.  One row group of G threads per (pair, row).
template <int N>
__global__ void k_c2r(const V* __restrict__ spec, float* __restrict__ phys, const V* __restrict__ tw, int F,
                      long long rows) {
  constexpr int E = EOf<float, N>::v, G = N / E, NH = N / 2 + 1;
  constexpr int RPC = 256 / G > 0 ? 256 / G : 1;
  extern __shared__ __align__(128) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int j0 = threadIdx.x % G, rl = threadIdx.x / G;
  const long long row = (long long)blockIdx.x * RPC + rl;
  const int f0 = 2 * blockIdx.y, f1 = f0 + 1;
  const bool ok = row < rows, has1 = f1 < F;
  RowExchange<V> ex{sm + rl * N, RPC * N, 0};
  const V* pa = spec + ((long long)f0 * rows + (ok ? row : 0)) * NH;
  const V* pb = spec + ((long long)(has1 ? f1 : f0) * rows + (ok ? row : 0)) * NH;
  V x[E];
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int n = j0 + m * (N / E);
    const bool hi = n > N / 2;
    const int p = hi ? N - n : n;
    V A = ok ? pa[p] : czero<V>(), B = (ok && has1) ? pb[p] : czero<V>();
    if (hi) {
      A = cconj(A);
      B = cconj(B);
    }
    x[m] = mk<V>(A.x - B.y, A.y + B.x);  // A + i B
  }
  line_fft<N, E, +1>(x, j0, tw, ex);
  if (ok) {
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int n = j0 + m * (N / E);
      phys[((long long)f0 * rows + row) * N + n] = x[m].x;
      if (has1) phys[((long long)f1 * rows + row) * N + n] = x[m].y;
    }
  }
}

template <int N>
__global__ void k_r2c(const float* __restrict__ phys, V* __restrict__ spec, const V* __restrict__ tw, int F,
                      long long rows, float scale) {
  constexpr int E = EOf<float, N>::v, G = N / E, NH = N / 2 + 1;
  constexpr int RPC = 256 / G > 0 ? 256 / G : 1;
  extern __shared__ __align__(128) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const int j0 = threadIdx.x % G, rl = threadIdx.x / G;
  const long long row = (long long)blockIdx.x * RPC + rl;
  const int f0 = 2 * blockIdx.y, f1 = f0 + 1;
  const bool ok = row < rows, has1 = f1 < F;
  RowExchange<V> ex{sm + rl * N, RPC * N, 0};
  V x[E];
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int n = j0 + m * (N / E);
    const float a = ok ? phys[((long long)f0 * rows + row) * N + n] : 0.f;
    const float b = (ok && has1) ? phys[((long long)f1 * rows + row) * N + n] : 0.f;
    x[m] = make_float2(a, b);
  }
  line_fft<N, E, -1>(x, j0, tw, ex);
#pragma unroll
  for (int m = 0; m < E; ++m) ex.put(j0 + m * (N / E), x[m]);
  ex.sync();
  if (ok) {
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int k = j0 + m * (N / E);
      if (k < NH) {
        const V Fk = x[m];
        const V Fm = cconj(ex.get(k == 0 ? 0 : N - k));
        spec[((long long)f0 * rows + row) * NH + k] = cscale(cadd(Fk, Fm), 0.5f * scale);
        if (has1) spec[((long long)f1 * rows + row) * NH + k] = cscale(cmul_mi(csub(Fk, Fm)), 0.5f * scale);
      }
    }
  }
}

template <int N, int DIR>
cudaError_t c2c_n(V* data, const V* tw, int ncols, int nb2, long long s1, long long s2, long long es, int nbatch,
                  cudaStream_t s) {
  constexpr int E = EOf<float, N>::v, G = N / E;
  constexpr int NBG = 256 / (TXG * G) > 0 ? 256 / (TXG * G) : 1;
  const size_t smem = 2ull * NBG * N * TXG * sizeof(V);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_c2c<N, DIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((ncols + TXG - 1) / TXG, (nbatch + NBG - 1) / NBG);
  k_c2c<N, DIR><<<grid, TXG * G * NBG, smem, s>>>(data, tw, ncols, nb2, s1, s2, es, nbatch);
  return cudaGetLastError();
}

template <int N>
cudaError_t c2r_n(const V* spec, float* phys, const V* tw, int F, long long rows, cudaStream_t s) {
  constexpr int E = EOf<float, N>::v, G = N / E;
  constexpr int RPC = 256 / G > 0 ? 256 / G : 1;
  const size_t smem = 2ull * RPC * N * sizeof(V);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_c2r<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((unsigned)((rows + RPC - 1) / RPC), (F + 1) / 2);
  k_c2r<N><<<grid, RPC * G, smem, s>>>(spec, phys, tw, F, rows);
  return cudaGetLastError();
}

template <int N>
cudaError_t r2c_n(const float* phys, V* spec, const V* tw, int F, long long rows, float scale, cudaStream_t s) {
  constexpr int E = EOf<float, N>::v, G = N / E;
  constexpr int RPC = 256 / G > 0 ? 256 / G : 1;
  const size_t smem = 2ull * RPC * N * sizeof(V);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_r2c<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((unsigned)((rows + RPC - 1) / RPC), (F + 1) / 2);
  k_r2c<N><<<grid, RPC * G, smem, s>>>(phys, spec, tw, F, rows, scale);
  return cudaGetLastError();
}

#define LES_DISPATCH(n, CALL)                  \
  switch (n) {                                 \
    case 16: return CALL(16);                  \
    case 32: return CALL(32);                  \
    case 48: return CALL(48);                  \
    case 64: return CALL(64);                  \
    case 96: return CALL(96);                  \
    case 128: return CALL(128);                \
    case 192: return CALL(192);                \
    case 256: return CALL(256);                \
    case 512: return CALL(512);                \
    default: return cudaErrorInvalidValue;     \
  }

cudaError_t c2c(int n, int dir, V* d, const V* tw, int ncols, int nb2, long long s1, long long s2, long long es,
                int nbatch, cudaStream_t s) {
  if (dir > 0) {
#define CALL(N) c2c_n<N, +1>(d, tw, ncols, nb2, s1, s2, es, nbatch, s)
    LES_DISPATCH(n, CALL)
#undef CALL
  } else {
#define CALL(N) c2c_n<N, -1>(d, tw, ncols, nb2, s1, s2, es, nbatch, s)
    LES_DISPATCH(n, CALL)
#undef CALL
  }
}
cudaError_t c2r(int n, const V* spec, float* phys, const V* tw, int F, long long rows, cudaStream_t s) {
#define CALL(N) c2r_n<N>(spec, phys, tw, F, rows, s)
  LES_DISPATCH(n, CALL)
#undef CALL
}
cudaError_t r2c(int n, const float* phys, V* spec, const V* tw, int F, long long rows, float scale,
                cudaStream_t s) {
#define CALL(N) r2c_n<N>(phys, spec, tw, F, rows, scale, s)
  LES_DISPATCH(n, CALL)
#undef CALL
}

// Spectral [F][nz][ny][nh] (overwritten by the z and y passes) -> physical
// [F][nz][ny][nx], unnormalised backward sum.
cudaError_t spec2phys(const Geo& g, int F, V* spec, float* phys, const V* twx, const V* twy, const V* twz,
                      cudaStream_t s) {
  const long long plane = (long long)g.ny * g.nh, fs = (long long)g.nz * plane;
  cudaError_t e = c2c(g.nz, +1, spec, twz, g.nh, g.ny, fs, g.nh, plane, F * g.ny, s);
  if (e == cudaSuccess) e = c2c(g.ny, +1, spec, twy, g.nh, g.nz, fs, plane, g.nh, F * g.nz, s);
  if (e == cudaSuccess) e = c2r(g.nx, spec, phys, twx, F, (long long)g.nz * g.ny, s);
  return e;
}

// Physical -> spectral with the 1/(nx ny nz) of the forward transform.
cudaError_t phys2spec(const Geo& g, int F, const float* phys, V* spec, const V* twx, const V* twy, const V* twz,
                      cudaStream_t s) {
  const long long plane = (long long)g.ny * g.nh, fs = (long long)g.nz * plane;
  const float scale = (float)(1.0 / ((double)g.nx * g.ny * g.nz));
  cudaError_t e = r2c(g.nx, phys, spec, twx, F, (long long)g.nz * g.ny, scale, s);
  if (e == cudaSuccess) e = c2c(g.ny, -1, spec, twy, g.nh, g.nz, fs, plane, g.nh, F * g.nz, s);
  if (e == cudaSuccess) e = c2c(g.nz, -1, spec, twz, g.nh, g.ny, fs, g.nh, plane, F * g.ny, s);
  return e;
}

// A_ij = i k_j u_i for kept modes (0 elsewhere), 9 fields [i][j] in the full
// spectral layout.
__global__ void k_grad(const Geo g, const Spec u, V* out) {
  const long long total = (long long)g.nz * g.ny * g.nh;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int p = (int)(i % g.nh), qi = (int)((i / g.nh) % g.ny), ri = (int)(i / ((long long)g.nh * g.ny));
  const int q = sidx(qi, g.ny), r = sidx(ri, g.nz);
  V uu[3] = {czero<V>(), czero<V>(), czero<V>()};
  if (kept(g, p, q, r)) {
    const V* pm = static_cast<const V*>(u.p) + (long long)rowof(r, u.zwrap) * u.zs +
                  (long long)rowof(q, u.ywrap) * u.ys + p;
    uu[0] = pm[0];
    uu[1] = pm[u.cs];
    uu[2] = pm[2 * u.cs];
  }
  const float k[3] = {float(p) * g.sxf, float(q) * g.syf, float(r) * g.szf};
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) out[(3 * a + b) * total + i] = cmul_i(cscale(uu[a], k[b]));
}

// Invariants tr S^2, tr R^2, tr S^3, tr S R^2, tr S^2 R^2 of A (9 physical
// fields), standardised: X[p][n] = (lambda_n - mean_n) * invstd_n, with
// norm = [mean 5 | invstd 5 | s_tau | 1/s_A].  Aout (optional) receives the
// gradient as rows [p][9].
__global__ void k_features(const float* __restrict__ A, float* __restrict__ X, float* __restrict__ Aout,
                           long long P, const float* __restrict__ norm) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= P) return;
  float a[3][3], S[3][3], R[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) a[i][j] = A[(3 * i + j) * P + p];
  if (Aout) {
#pragma unroll
    for (int k = 0; k < 9; ++k) Aout[p * 9 + k] = a[k / 3][k % 3];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      S[i][j] = 0.5f * (a[i][j] + a[j][i]);
      R[i][j] = 0.5f * (a[i][j] - a[j][i]);
    }
  float S2[3][3], R2[3][3];
  matmul3(S, S, S2);
  matmul3(R, R, R2);
  float l1 = 0, l2 = 0, l3 = 0, l4 = 0, l5 = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    l1 += S2[i][i];
    l2 += R2[i][i];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      l3 += S2[i][k] * S[k][i];
      l4 += S[i][k] * R2[k][i];
      l5 += S2[i][k] * R2[k][i];
    }
  }
  const float lam[5] = {l1, l2, l3, l4, l5};
#pragma unroll
  for (int n = 0; n < 5; ++n) X[p * 5 + n] = (lam[n] - norm[n]) * norm[5 + n];
}

// Model stress tau = s_tau sum_n Y[p][n] T_n(A/s_A), written over fields 0..5
// of the gradient buffer G (9 planar fields; each point reads its own nine
// values before writing six, so no __restrict__).
__global__ void k_stress(float* G, const float* __restrict__ Y, long long P, const float* __restrict__ norm) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= P) return;
  float a[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) a[i][j] = G[(3 * i + j) * P + p];
  float Tb[6][6];
  tensor_basis(a, norm[11], Tb);
  float g[6];
#pragma unroll
  for (int n = 0; n < 6; ++n) g[n] = Y[p * 6 + n];
  const float st = norm[10];
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    float t = 0.f;
#pragma unroll
    for (int n = 0; n < 6; ++n) t += g[n] * Tb[n][m];
    G[m * P + p] = st * t;
  }
}

// extra_c = -i sum_j k_j tau_hat_cj for kept modes, compact layout.
__global__ void k_div(const Geo g, const V* __restrict__ th, V* __restrict__ extra) {
  const long long total = (long long)g.cz * g.cy * g.cx;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int p = (int)(i % g.cx), iy = (int)((i / g.cx) % g.cy), iz = (int)(i / ((long long)g.cx * g.cy));
  const int q = iy <= g.Ky ? iy : iy - g.cy, r = iz <= g.Kz ? iz : iz - g.cz;
  const long long ci = ((long long)iz * g.cy + iy) * g.kxp + p, cs = (long long)g.cz * g.cy * g.kxp;
  if (!kept(g, p, q, r)) {
    for (int c = 0; c < 3; ++c) extra[c * cs + ci] = czero<V>();
    return;
  }
  const long long fs = (long long)g.nz * g.ny * g.nh;
  const long long fi = ((long long)rowof(r, g.nz) * g.ny + rowof(q, g.ny)) * g.nh + p;
  const float k[3] = {float(p) * g.sxf, float(q) * g.syf, float(r) * g.szf};
  // symmetric components in the order 11, 22, 33, 12, 13, 23
  const int idx[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    V s = czero<V>();
#pragma unroll
    for (int j = 0; j < 3; ++j) s = cadd(s, cscale(th[idx[c][j] * fs + fi], k[j]));
    extra[c * cs + ci] = cmul_mi(s);  // -i s
  }
}

// r_hat = D P(extra) - f for the full-layout modes (zero outside the kept
// set), loss += sum w |r_hat|^2 (w = 1 on the kx = 0 plane, else 2).
__global__ void k_force_residual(const Geo g, const V* __restrict__ extra, const Spec f, V* __restrict__ rh,
                                 double* loss) {
  __shared__ double red[32];
  const long long total = (long long)g.nz * g.ny * g.nh;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(i % g.nh), qi = (int)((i / g.nh) % g.ny), ri = (int)(i / ((long long)g.nh * g.ny));
    const int q = sidx(qi, g.ny), r = sidx(ri, g.nz);
    V o[3] = {czero<V>(), czero<V>(), czero<V>()};
    if (kept(g, p, q, r)) {
      const long long cs = (long long)g.cz * g.cy * g.kxp;
      const long long ci = ((long long)rowof(r, g.cz) * g.cy + rowof(q, g.cy)) * g.kxp + p;
      V v[3] = {extra[ci], extra[ci + cs], extra[ci + 2 * cs]};
      const float kx = float(p) * g.sxf, ky = float(q) * g.syf, kz = float(r) * g.szf;
      const float k2 = kx * kx + ky * ky + kz * kz;
      if (k2 > 0.f) {
        const V kd = cadd(cadd(cscale(v[0], kx), cscale(v[1], ky)), cscale(v[2], kz));
        const float ik2 = 1.f / k2;
        v[0] = csub(v[0], cscale(kd, kx * ik2));
        v[1] = csub(v[1], cscale(kd, ky * ik2));
        v[2] = csub(v[2], cscale(kd, kz * ik2));
      } else {
        v[0] = v[1] = v[2] = czero<V>();
      }
      const V* fp = static_cast<const V*>(f.p) + (long long)rowof(r, f.zwrap) * f.zs +
                    (long long)rowof(q, f.ywrap) * f.ys + p;
      const double w = p == 0 ? 1.0 : 2.0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        o[c] = csub(v[c], fp[c * f.cs]);
        acc += w * ((double)o[c].x * o[c].x + (double)o[c].y * o[c].y);
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) rh[c * total + i] = o[c];
  }
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0) atomicAdd(loss, t);
}

// Shell energy transfer of the projected closure term: bins[K] +=
// w Re(u* . D P extra) over the kept modes, K = floor(|k| + 1/2) < nsh.
__global__ void k_transfer_shells(const Geo g, const V* __restrict__ extra, const Spec u, double* bins, int nsh) {
  extern __shared__ double sb[];
  for (int i = threadIdx.x; i < nsh; i += blockDim.x) sb[i] = 0.0;
  __syncthreads();
  const long long total = (long long)g.cz * g.cy * g.cx;
  const long long cs = (long long)g.cz * g.cy * g.kxp;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(i % g.cx), iy = (int)((i / g.cx) % g.cy), iz = (int)(i / ((long long)g.cx * g.cy));
    const int q = iy <= g.Ky ? iy : iy - g.cy, r = iz <= g.Kz ? iz : iz - g.cz;
    if (!kept(g, p, q, r)) continue;
    const double kx = p * g.sx, ky = q * g.sy, kz = r * g.sz;
    const int K = (int)floor(sqrt(kx * kx + ky * ky + kz * kz) + 0.5);
    if (K >= nsh) continue;
    const long long ci = ((long long)iz * g.cy + iy) * g.kxp + p;
    double v[3][2] = {{extra[ci].x, extra[ci].y}, {extra[ci + cs].x, extra[ci + cs].y},
                      {extra[ci + 2 * cs].x, extra[ci + 2 * cs].y}};
    const double k2 = kx * kx + ky * ky + kz * kz;
    if (k2 > 0) {
      const double dr = (kx * v[0][0] + ky * v[1][0] + kz * v[2][0]) / k2;
      const double di = (kx * v[0][1] + ky * v[1][1] + kz * v[2][1]) / k2;
      const double kk[3] = {kx, ky, kz};
      for (int c = 0; c < 3; ++c) {
        v[c][0] -= kk[c] * dr;
        v[c][1] -= kk[c] * di;
      }
    } else {
      continue;
    }
    const V* up = static_cast<const V*>(u.p) + (long long)rowof(r, u.zwrap) * u.zs + (long long)rowof(q, u.ywrap) * u.ys + p;
    double e = 0.0;
    for (int c = 0; c < 3; ++c) {
      const V a = up[c * u.cs];
      e += (double)a.x * v[c][0] + (double)a.y * v[c][1];
    }
    atomicAdd(sb + K, (p == 0 ? 1.0 : 2.0) * e);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nsh; i += blockDim.x) atomicAdd(bins + i, sb[i]);
}

// dT = bins - T_exact, loss += sum dT^2 (one block).
__global__ void k_transfer_delta(const double* __restrict__ bins, const double* __restrict__ te, int nsh,
                                 double* __restrict__ dT, double* loss) {
  __shared__ double red[32];
  double a = 0.0;
  for (int i = threadIdx.x; i < nsh; i += blockDim.x) {
    const double d = bins[i] - te[i];
    dT[i] = d;
    a += d * d;
  }
  const double t = block_sum(a, red);
  if (threadIdx.x == 0) atomicAdd(loss, t);
}

// r_hat(k) = dT(K(k)) u(k) on the kept modes (full layout, zero elsewhere).
__global__ void k_transfer_residual(const Geo g, const Spec u, const double* __restrict__ dT, int nsh,
                                    V* __restrict__ rh) {
  const long long total = (long long)g.nz * g.ny * g.nh;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(i % g.nh), qi = (int)((i / g.nh) % g.ny), ri = (int)(i / ((long long)g.nh * g.ny));
    const int q = sidx(qi, g.ny), r = sidx(ri, g.nz);
    V o[3] = {czero<V>(), czero<V>(), czero<V>()};
    if (kept(g, p, q, r)) {
      const double kx = p * g.sx, ky = q * g.sy, kz = r * g.sz;
      const int K = (int)floor(sqrt(kx * kx + ky * ky + kz * kz) + 0.5);
      if (K < nsh) {
        const float d = (float)dT[K];
        const V* up = static_cast<const V*>(u.p) + (long long)rowof(r, u.zwrap) * u.zs +
                      (long long)rowof(q, u.ywrap) * u.ys + p;
        for (int c = 0; c < 3; ++c) o[c] = cscale(up[c * u.cs], d);
      }
    }
    for (int c = 0; c < 3; ++c) rh[c * total + i] = o[c];
  }
}

// dL/dg_n = s_tau sum_m T_n,m(A/s_A) dL/dtau_m with dL/dtau_ij = c d r_i/d x_j
// (both orders for an off-diagonal component); G holds d r_i / d x_j as 9
// planar fields [3i+j], Arows the gradient of the state.
__global__ void k_dg(const float* __restrict__ Arows, const float* __restrict__ G, const float* __restrict__ norm,
                     float c, float* __restrict__ dY, long long P) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= P) return;
  float a[3][3];
#pragma unroll
  for (int k = 0; k < 9; ++k) a[k / 3][k % 3] = Arows[p * 9 + k];
  float Tb[6][6];
  tensor_basis(a, norm[11], Tb);
  const int ii[6] = {0, 1, 2, 0, 0, 1}, jj[6] = {0, 1, 2, 1, 2, 2};
  float dt[6];
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    const float gij = G[(3 * ii[m] + jj[m]) * P + p];
    dt[m] = c * (m < 3 ? gij : gij + G[(3 * jj[m] + ii[m]) * P + p]);
  }
  const float st = norm[10];
#pragma unroll
  for (int n = 0; n < 6; ++n) {
    float v = 0.f;
#pragma unroll
    for (int m = 0; m < 6; ++m) v += Tb[n][m] * dt[m];
    dY[p * 6 + n] = st * v;
  }
}

}  // namespace les

cudaError_t les_closure_term(const Geo& g, Spec in, const void* twx, const void* twy, const void* twz,
                             const LesScratch& s, cudaStream_t st) {
  using namespace les;
  const long long P = (long long)g.nx * g.ny * g.nz;
  const long long M = (long long)g.nz * g.ny * g.nh;
  const V *tx = static_cast<const V*>(twx), *ty = static_cast<const V*>(twy), *tz = static_cast<const V*>(twz);
  k_grad<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(g, in, s.spec);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = spec2phys(g, 9, s.spec, s.phys, tx, ty, tz, st);
  if (e == cudaSuccess) {
    k_features<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(s.phys, s.X, nullptr, P, s.norm);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    const ps_status ms = ps_mlp_forward(s.params, s.X, s.Y, P, st);
    if (ms != PS_OK) return cudaErrorLaunchFailure;
  }
  if (e == cudaSuccess) {
    k_stress<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(s.phys, s.Y, P, s.norm);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = phys2spec(g, 6, s.phys, s.spec, tx, ty, tz, st);
  if (e == cudaSuccess) {
    const long long C = (long long)g.cz * g.cy * g.cx;
    k_div<<<(unsigned)((C + 255) / 256), 256, 0, st>>>(g, s.spec, s.extra);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t les_closure_grad(const Geo& g, Spec in, Spec f, const void* twx, const void* twy, const void* twz,
                             const LesScratch& s, const float* params, float* grad, double* loss, cudaStream_t st,
                             const double* t_exact, int nsh, double* bins) {
  using namespace les;
  const long long P = (long long)g.nx * g.ny * g.nz;
  const long long M = (long long)g.nz * g.ny * g.nh;
  const V *tx = static_cast<const V*>(twx), *ty = static_cast<const V*>(twy), *tz = static_cast<const V*>(twz);
  // forward: features (keeping the gradient rows), network, stress, its
  // divergence (compact), as in les_closure_term
  k_grad<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(g, in, s.spec);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = spec2phys(g, 9, s.spec, s.phys, tx, ty, tz, st);
  if (e == cudaSuccess) {
    k_features<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(s.phys, s.X, s.Arows, P, s.norm);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && ps_mlp_forward(params, s.X, s.Y, P, st) != PS_OK) e = cudaErrorLaunchFailure;
  if (e == cudaSuccess) {
    k_stress<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(s.phys, s.Y, P, s.norm);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = phys2spec(g, 6, s.phys, s.spec, tx, ty, tz, st);
  if (e == cudaSuccess) {
    const long long C = (long long)g.cz * g.cy * g.cx;
    k_div<<<(unsigned)((C + 255) / 256), 256, 0, st>>>(g, s.spec, s.extra);
    e = cudaGetLastError();
  }
  // residual and loss; d r_i / d x_j (k_grad reads each mode's three values
  // before writing its nine, so it runs in place on the spectral buffer)
  if (e == cudaSuccess && !t_exact) {
    k_force_residual<<<1024, 256, 0, st>>>(g, s.extra, f, s.spec, loss);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && t_exact) {
    // transfer loss: bins = T_model, dT = bins - T_exact (in bins + nsh)
    e = cudaMemsetAsync(bins, 0, sizeof(double) * nsh, st);
    if (e == cudaSuccess) {
      k_transfer_shells<<<256, 256, sizeof(double) * nsh, st>>>(g, s.extra, in, bins, nsh);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      k_transfer_delta<<<1, 128, 0, st>>>(bins, t_exact, nsh, bins + nsh, loss);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      k_transfer_residual<<<1024, 256, 0, st>>>(g, in, bins + nsh, nsh, s.spec);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) {
    Spec r;
    r.p = s.spec;
    r.ys = g.nh;
    r.zs = (long long)g.ny * g.nh;
    r.cs = M;
    r.zwrap = g.nz;
    r.ywrap = g.ny;
    k_grad<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(g, r, s.spec);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = spec2phys(g, 9, s.spec, s.phys, tx, ty, tz, st);
  // adjoint through the tensor basis, then the network
  if (e == cudaSuccess) {
    k_dg<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(s.Arows, s.phys, s.norm, (float)(2.0 / (double)P), s.Y, P);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && ps_mlp_backward(params, s.X, s.Y, P, grad, st) != PS_OK) e = cudaErrorLaunchFailure;
  return e;
}

namespace les {

// Rows T[p][m] of 6 planar physical fields.
__global__ void k_rows6(const float* __restrict__ f, float* __restrict__ T, long long P) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= P) return;
#pragma unroll
  for (int m = 0; m < 6; ++m) T[p * 6 + m] = f[m * P + p];
}

// u_i u_j (order 11, 22, 33, 12, 13, 23) of 3 planar fields u into 6 fields uu;
// may run in place with u = uu + 3P (each point reads its three values first).
__global__ void k_products(const float* u, float* uu, long long P) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= P) return;
  const float a = u[p], b = u[P + p], c = u[2 * P + p];
  uu[p] = a * a;
  uu[P + p] = b * b;
  uu[2 * P + p] = c * c;
  uu[3 * P + p] = a * b;
  uu[4 * P + p] = a * c;
  uu[5 * P + p] = b * c;
}

// Copy the modes |p|,|q|,|r| <= kc of F full-layout fields on grid gs into
// grid gd (zeros elsewhere).
__global__ void k_truncate(const V* __restrict__ src, const Geo gs, V* __restrict__ dst, const Geo gd, int kc, int F) {
  const long long td = (long long)gd.nz * gd.ny * gd.nh;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= td * F) return;
  const int f = (int)(i / td);
  const long long j = i % td;
  const int p = (int)(j % gd.nh), qi = (int)((j / gd.nh) % gd.ny), ri = (int)(j / ((long long)gd.nh * gd.ny));
  const int q = sidx(qi, gd.ny), r = sidx(ri, gd.nz);
  V v = czero<V>();
  if (p <= kc && q <= kc && q >= -kc && r <= kc && r >= -kc) {
    const long long ts = (long long)gs.nz * gs.ny * gs.nh;
    v = src[f * ts + ((long long)rowof(r, gs.nz) * gs.ny + rowof(q, gs.ny)) * gs.nh + p];
  }
  dst[i] = v;
}

// a <- a - b on F fields of one grid (full layout).
__global__ void k_sub(V* __restrict__ a, const V* __restrict__ b, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) a[i] = csub(a[i], b[i]);
}

Geo cube_geo(int n) {
  Geo g{};
  g.nx = g.ny = g.nz = n;
  g.nh = n / 2 + 1;
  g.Kx = g.Ky = g.Kz = (n + 2) / 3 - 1;
  g.cx = g.Kx + 1;
  g.cy = g.cz = 2 * g.Kx + 1;
  g.kxp = (g.cx + 15) / 16 * 16;
  set_scales(g, 6.283185307179586476925286766559, 6.283185307179586476925286766559,
             6.283185307179586476925286766559);  // 2 pi box
  return g;
}

unsigned blocks(long long n) { return (unsigned)((n + 255) / 256); }

}  // namespace les
}  // namespace ps

extern "C" ps_status ps_les_training_sample(int n_dns, const void* uhat_dns, int n_les, int kc, const double* norm12,
                                            float* X, float* A, float* T, void* cuda_stream) {
  using namespace ps;
  using namespace ps::les;
  auto bad = [](const char* m) {
    set_last_error(m);
    return PS_ERR_INVALID_ARG;
  };
  auto ok_n = [](int n) {
    return n == 16 || n == 32 || n == 48 || n == 64 || n == 96 || n == 128 || n == 192 || n == 256 || n == 512;
  };
  if (!uhat_dns || !X || !T) return bad("ps_les_training_sample: NULL buffer");
  if (!ok_n(n_dns) || !ok_n(n_les) || n_les > n_dns) return bad("ps_les_training_sample: unsupported grid sizes");
  if (kc < 1 || kc > (n_les + 2) / 3 - 1) return bad("ps_les_training_sample: kc must be in 1..ceil(n_les/3)-1");
  if (norm12)
    for (int i = 5; i < 10; ++i)
      if (!(norm12[i] > 0) || !std::isfinite(norm12[i])) return bad("ps_les_training_sample: std must be positive");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const Geo gd = cube_geo(n_dns), gl = cube_geo(n_les);
  const long long Md = (long long)gd.nz * gd.ny * gd.nh, Pd = (long long)n_dns * n_dns * n_dns;
  const long long Ml = (long long)gl.nz * gl.ny * gl.nh, Pl = (long long)n_les * n_les * n_les;
  std::vector<void*> bufs;
  auto alloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    bufs.push_back(p);
    return p;
  };
  V* twd = static_cast<V*>(alloc(sizeof(V) * n_dns));
  V* twl = static_cast<V*>(alloc(sizeof(V) * n_les));
  V* sd = static_cast<V*>(alloc(sizeof(V) * 6 * Md));              // DNS spectra (6 fields)
  float* pd = static_cast<float*>(alloc(sizeof(float) * 6 * Pd));  // DNS physical (6 fields)
  V* sl = static_cast<V*>(alloc(sizeof(V) * 6 * Ml));              // LES spectra (6 fields)
  V* sg = static_cast<V*>(alloc(sizeof(V) * 9 * Ml));              // LES spectra (9 fields)
  float* pl = static_cast<float*>(alloc(sizeof(float) * 9 * Pl));  // LES physical (9 fields)
  float* nrm = static_cast<float*>(alloc(sizeof(float) * 12));
  ps_status st = PS_OK;
  if (!twd || !twl || !sd || !pd || !sl || !sg || !pl || !nrm) {
    set_last_error("ps_les_training_sample: device allocation failed");
    st = PS_ERR_OOM;
  }
  cudaError_t e = cudaSuccess;
  const unsigned bd = blocks(Pd), bl = blocks(Pl);
  const size_t ubytes = sizeof(V) * 3 * Md;
  if (st == PS_OK) {
    float h[12];
    for (int i = 0; i < 5; ++i) {
      h[i] = norm12 ? (float)norm12[i] : 0.f;
      h[5 + i] = norm12 ? (float)(1.0 / norm12[5 + i]) : 1.f;
    }
    h[10] = h[11] = 1.f;
    e = cudaMemcpyAsync(nrm, h, sizeof(h), cudaMemcpyHostToDevice, s);
    k_tw<<<(n_dns + 255) / 256, 256, 0, s>>>(twd, n_dns);
    k_tw<<<(n_les + 255) / 256, 256, 0, s>>>(twl, n_les);
    // 1. F[u_i u_j] on the LES grid: DNS velocity (fields 3..5 of pd), the
    //    products in place, forward, truncate
    if (e == cudaSuccess) e = cudaMemcpyAsync(sd, uhat_dns, ubytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = spec2phys(gd, 3, sd, pd + 3 * Pd, twd, twd, twd, s);
    if (e == cudaSuccess) {
      k_products<<<bd, 256, 0, s>>>(pd + 3 * Pd, pd, Pd);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = phys2spec(gd, 6, pd, sd, twd, twd, twd, s);
    if (e == cudaSuccess) {
      k_truncate<<<blocks(6 * Ml), 256, 0, s>>>(sd, gd, sl, gl, kc, 6);
      e = cudaGetLastError();
    }
    // 2. F[ubar_i ubar_j]: ubar on the LES grid (3 < 2/3 of the grid, so its
    //    products do not alias below kc), products, forward, truncate
    if (e == cudaSuccess) e = cudaMemcpyAsync(sd, uhat_dns, ubytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) {
      k_truncate<<<blocks(3 * Ml), 256, 0, s>>>(sd, gd, sg, gl, kc, 3);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = spec2phys(gl, 3, sg, pl + 3 * Pl, twl, twl, twl, s);
    if (e == cudaSuccess) {
      k_products<<<bl, 256, 0, s>>>(pl + 3 * Pl, pl, Pl);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = phys2spec(gl, 6, pl, sg, twl, twl, twl, s);
    if (e == cudaSuccess) {
      k_sub<<<blocks(6 * Ml), 256, 0, s>>>(sl, sg, 6 * Ml);
      e = cudaGetLastError();
    }
    // 3. tau = F[uu] - F[ubar ubar]: truncate the difference, back to the LES grid
    if (e == cudaSuccess) {
      k_truncate<<<blocks(6 * Ml), 256, 0, s>>>(sl, gl, sg, gl, kc, 6);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = spec2phys(gl, 6, sg, pl, twl, twl, twl, s);
    if (e == cudaSuccess) {
      k_rows6<<<bl, 256, 0, s>>>(pl, T, Pl);
      e = cudaGetLastError();
    }
    // 4. features of grad ubar
    if (e == cudaSuccess) e = cudaMemcpyAsync(sd, uhat_dns, ubytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) {
      k_truncate<<<blocks(3 * Ml), 256, 0, s>>>(sd, gd, sl, gl, kc, 3);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      Spec in;
      in.p = sl;
      in.ys = gl.nh;
      in.zs = (long long)gl.ny * gl.nh;
      in.cs = (long long)gl.nz * gl.ny * gl.nh;
      in.zwrap = gl.nz;
      in.ywrap = gl.ny;
      Geo gk = gl;
      gk.Kx = gk.Ky = gk.Kz = kc;
      k_grad<<<blocks(Ml), 256, 0, s>>>(gk, in, sg);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = spec2phys(gl, 9, sg, pl, twl, twl, twl, s);
    if (e == cudaSuccess) {
      k_features<<<bl, 256, 0, s>>>(pl, X, A, Pl, nrm);
      e = cudaGetLastError();
    }
  }
  if (st == PS_OK && e != cudaSuccess) {
    set_last_error(std::string("ps_les_training_sample: ") + cudaGetErrorString(e));
    st = PS_ERR_CUDA;
  }
  cudaStreamSynchronize(s);
  for (void* b : bufs) cudaFree(b);
  return st;
}

extern "C" ps_status ps_les_filter(int n_dns, const void* uhat_dns, int n_les, int kc, void* uhat_les,
                                   void* cuda_stream) {
  using namespace ps;
  using namespace ps::les;
  if (!uhat_dns || !uhat_les) {
    set_last_error("ps_les_filter: NULL buffer");
    return PS_ERR_INVALID_ARG;
  }
  const auto ok_n = [](int n) { return n >= 8 && n <= 1024 && n % 2 == 0; };
  if (!ok_n(n_dns) || !ok_n(n_les) || n_les > n_dns || kc < 0 || 2 * kc >= n_les) {
    set_last_error("ps_les_filter: need even sizes 8..1024, n_les <= n_dns and 0 <= kc < n_les/2");
    return PS_ERR_INVALID_ARG;
  }
  if (uhat_dns == uhat_les) {
    set_last_error("ps_les_filter: input and output may not alias");
    return PS_ERR_INVALID_ARG;
  }
  const Geo gd = cube_geo(n_dns), gl = cube_geo(n_les);
  const long long Ml = (long long)gl.nz * gl.ny * gl.nh;
  k_truncate<<<blocks(3 * Ml), 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
      static_cast<const V*>(uhat_dns), gd, static_cast<V*>(uhat_les), gl, kc, 3);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string("ps_les_filter: ") + cudaGetErrorString(e));
    return PS_ERR_CUDA;
  }
  return PS_OK;
}

// Plain 3D transforms of FP32 fields (include/ps.h, ps_fft_c2r / ps_fft_r2c):
// the line transforms of the passes without pruning, masking or fusion.
namespace {

ps_status fft_bad(ps_status s, const std::string& m) {
  ps::set_last_error(m);
  return s;
}

ps_status fft_run(int n, int nfields, const void* in, void* out, void* cuda_stream, bool backward) {
  using namespace ps;
  using namespace ps::les;
  const char* name = backward ? "ps_fft_c2r" : "ps_fft_r2c";
  const auto ok_n = [](int v) {
    return v == 16 || v == 32 || v == 48 || v == 64 || v == 96 || v == 128 || v == 192 || v == 256 || v == 512;
  };
  if (!in || !out) return fft_bad(PS_ERR_INVALID_ARG, std::string(name) + ": NULL buffer");
  if (!ok_n(n)) return fft_bad(PS_ERR_INVALID_ARG, std::string(name) + ": n must be 16, 32, 48, 64, 96, 128, 192, 256 or 512");
  if (nfields < 1 || nfields > 16) return fft_bad(PS_ERR_INVALID_ARG, std::string(name) + ": nfields must be in 1..16");
  const Geo g = cube_geo(n);
  const long long M = (long long)g.nz * g.ny * g.nh, P = (long long)n * n * n;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  V* tw = nullptr;
  V* spec = nullptr;
  cudaError_t e = cudaMalloc(&tw, sizeof(V) * n);
  if (e == cudaSuccess && backward) e = cudaMalloc(&spec, sizeof(V) * nfields * M);  // the z, y passes work in place
  if (e != cudaSuccess) {
    cudaFree(tw);
    (void)cudaGetLastError();
    return fft_bad(PS_ERR_OOM, std::string(name) + ": device allocation failed");
  }
  k_tw<<<(n + 255) / 256, 256, 0, s>>>(tw, n);
  e = cudaGetLastError();
  if (backward) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(spec, in, sizeof(V) * nfields * M, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = spec2phys(g, nfields, spec, static_cast<float*>(out), tw, tw, tw, s);
  } else {
    if (e == cudaSuccess) e = phys2spec(g, nfields, static_cast<const float*>(in), static_cast<V*>(out), tw, tw, tw, s);
  }
  const cudaError_t es = cudaStreamSynchronize(s);  // the scratch is freed below
  if (e == cudaSuccess) e = es;
  cudaFree(tw);
  cudaFree(spec);
  (void)P;
  if (e != cudaSuccess) return fft_bad(PS_ERR_CUDA, std::string(name) + ": " + cudaGetErrorString(e));
  return PS_OK;
}

}  // namespace

extern "C" ps_status ps_fft_c2r(int n, int nfields, const void* spec, float* phys, void* cuda_stream) {
  return fft_run(n, nfields, spec, phys, cuda_stream, true);
}

extern "C" ps_status ps_fft_r2c(int n, int nfields, const float* phys, void* spec, void* cuda_stream) {
  return fft_run(n, nfields, phys, spec, cuda_stream, false);
}
