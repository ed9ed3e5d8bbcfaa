// The five passes of one right-hand-side evaluation (Sec. 2 of the paper: the
// nonlinear term is formed in physical space between a backward and a forward
// 3D transform, and the pressure projects it onto divergence-free fields;
// Sec. 2 also describes each 3D transform as per-axis 1D transforms with a
// transpose between them).
//
//   zinv : u_hat (3 fields, retained modes) -> curl in registers -> backward
//          transform along z of u and omega (6 fields)            [a6]
//   yinv : backward transform along y                              [a6 -> b6]
//   xpass: per (z,y) row, backward transform along x of u + i omega (3 complex
//          lines), n = u x omega pointwise, forward transform of n_x + i n_y and
//          n_z, split, keep kx <= Kx                               [b6 -> a6]
//   yfwd : forward transform along y, keep |ky| <= Ky               [a6 -> b6]
//   zfwd : forward transform along z, keep |kz| <= Kz, 1/(Nx Ny Nz), forcing,
//          Leray projection, and the right-hand side or the integrating-factor
//          Runge-Kutta stage update                                 [b6 -> out]
//
// Only the retained 2/3-rule cube |p|<=Kx, |q|<=Ky, |r|<=Kz is ever read or
// transformed where the input is known to vanish elsewhere (pruned transforms);
// the result is identical to full transforms of the masked field.
#pragma once
#include <type_traits>
#include "ps_async.cuh"
#include "ps_fft.cuh"
#include "ps_kernels.h"

namespace ps {

// kx columns per CTA in the strided passes: 64-byte row segments
#ifndef PS_TX32
#define PS_TX32 8
#endif
// (K names the pass: 0 z-inverse, 1 y passes, 2 z-forward.  Segments of 32 B
// (4 columns) and 128 B (16 columns) measured slower in every strided pass.)
template <typename T, int K = 0> struct TXOf {
  static constexpr int v = sizeof(T) == 4 ? PS_TX32 : 4;
};
// Points per thread of pass K (0 z-inverse, 1 y passes, 2 z-forward, 3 x
// pass).  At 1024 points FP32 every pass takes 16 (three stages, two
// exchanges per line); the x pass then needs 231 registers and runs
// without spills at one CTA per SM (MinB below): 10.98 ms per 1024^3 launch,
// against 13.08 ms at 8 points per thread (four stages, three exchanges)
// and 14.70 ms at 16 points capped to 128 registers (spills).
template <typename T, int N, int K> struct EPass {
  static constexpr int v = EOf<T, N>::v;
};
// lines batched per CTA in the strided passes (about 256 threads per CTA)
template <typename T, int N, int K = 0> struct NBOf {
  static constexpr int G = N / EPass<T, N, K>::v;
  static constexpr int q = 256 / (TXOf<T, K>::v * G);
  static constexpr int v = q < 1 ? 1 : q;
};
template <typename T, int N, int K = 0> struct ColThreads {
  static constexpr int v = TXOf<T, K>::v * (N / EPass<T, N, K>::v) * NBOf<T, N, K>::v;
};
// Shape of column pass K (0 z-inverse, 1 y passes, 2 z-forward) on lines of
// N points: kx columns per CTA (TX), points per thread (E), threads per line
// (G), lines of the other index per CTA (NB, about 256 threads per CTA).
// VAR 0 is the default above; VAR 1 halves the columns per CTA (twice the
// lines); VAR 2 takes the other radix schedule, 8 <-> 16 points per thread
// (lengths with a factor 3 keep theirs).  Plans of the grids that the
// ensemble tuner shapes (HasShapes) carry the variant per pass.
template <typename T, int N> struct AltE {
  static constexpr int e0 = EOf<T, N>::v;
  static constexpr int v = (N % 3 == 0) ? e0 : e0 == 16 ? 8 : 16;
};
template <typename T, int N, int K, int VAR = 0> struct ColShape {
  static constexpr int TX = VAR == 1 ? TXOf<T, K>::v / 2 : TXOf<T, K>::v;
  static constexpr int E = VAR == 2 ? AltE<T, N>::v : EPass<T, N, K>::v;
  static constexpr int G = N / E;
  static constexpr int q = 256 / (TX * G);
  static constexpr int NB = q < 1 ? 1 : q;
  static constexpr int NTH = TX * G * NB;
};
template <typename T, int N> struct HasShapes {
  static constexpr bool v = sizeof(T) == 4 && (N == 64 || N == 96 || N == 128);
};

// rows per CTA in the x pass
template <typename T, int N> struct RPCOf {
  static constexpr int G = N / EPass<T, N, 3>::v;
  static constexpr int v = G >= 256 ? 1 : 256 / G;
};

// x pass: per-thread twiddle table in shared memory when it takes at most 8 KB
template <typename T, int N> struct XTwTable {
  static constexpr int E = EPass<T, N, 3>::v;
  static constexpr bool v = (size_t)TwSlots<N, E>::total * (N / E) * sizeof(typename cplx<T>::type) <= 8192;
};

// x pass: lines per row transformed together (exchange region of a row)
constexpr int XLINES = 3;

// x pass: twiddles in registers for the whole kernel when there are few
#ifndef PS_XTWREG
#define PS_XTWREG 14
#endif
template <typename T, int N> struct XTwReg {
  static constexpr int E = EPass<T, N, 3>::v;
  static constexpr bool v = sizeof(T) == 4 && E == 8 && TwSlots<N, E>::total <= PS_XTWREG;
};

// Minimum resident CTAs per SM requested from the register allocator.
#ifndef PS_XROWBAR
#define PS_XROWBAR 1
#endif
#ifndef PS_MINB_ZINV
#define PS_MINB_ZINV 2
#endif
#ifndef PS_MINB_XPASS
#define PS_MINB_XPASS 2
#endif
#ifndef PS_MINB_Y1024
#define PS_MINB_Y1024 2
#endif
#ifndef PS_MINB_ZF1024
#define PS_MINB_ZF1024 2
#endif
// Exchange buffers of the y passes and the z-forward pass: one (two barriers
// per exchange) for FP32 lines of 64 points and more, two (one barrier) else.
// The single buffer lets more CTAs share an SM: four of 512 threads at 512
// points (32 registers; 2 % faster than three CTAs with two buffers), two at
// 1024 points (64 registers; two buffers of 128 KB held the SM to one CTA:
// 1.3-1.4x slower), register-limited counts below (256^3 step 5 % faster).
#ifndef PS_COLBUF512
#define PS_COLBUF512 1
#endif
#ifndef PS_MINB_Y512
#define PS_MINB_Y512 4
#endif
#ifndef PS_MINB_ZF512
#define PS_MINB_ZF512 4
#endif
#ifndef PS_COLBUF_SMALL
#define PS_COLBUF_SMALL 1
#endif
#ifndef PS_COLBUF1024
#define PS_COLBUF1024 1
#endif
template <typename T, int N> struct ColBuf {
  static constexpr int v = sizeof(T) == 4 && N == 1024 ? PS_COLBUF1024 : sizeof(T) == 4 && N == 512 ? PS_COLBUF512
                           : sizeof(T) == 4 && N >= 64 ? PS_COLBUF_SMALL : 2;
};
// x pass: whether the launcher halves the rows per CTA to fit its shared
// memory (stage + exchange above 113 KB at RPCOf rows; kx extent of the
// 2/3 rule).  Its CTAs then have half the threads of the launch bound and
// two of them fill the SM's shared memory, so the kernel may use the
// registers of one full-size CTA per SM instead of spilling (FP32 256-point
// rows: 0.152 -> 0.135 ms per 256^3 launch; 1024-point rows: 13.08 ->
// 10.98 ms per 1024^3 launch).
template <typename T, int N> struct XHalved {
  static constexpr long long kxp = ((N + 2) / 3 + 15) / 16 * 16;
  static constexpr int E = EPass<T, N, 3>::v, R = RPCOf<T, N>::v;
  static constexpr long long tt =
      (!XTwReg<T, N>::v && XTwTable<T, N>::v) ? (long long)TwSlots<N, E>::total * (N / E) : 0;
  static constexpr long long bytes = (6LL * R * kxp + 3LL * R * N + tt) * (long long)sizeof(typename cplx<T>::type);
  static constexpr bool v = bytes > 113LL * 1024;
};
template <typename T, int N> struct MinB {
  // (1024-point z lines: the input tile and exchange hold one CTA per SM)
  static constexpr int zinv = N == 1024 ? 1 : PS_MINB_ZINV;
  static constexpr int xpass = XHalved<T, N>::v ? 1 : PS_MINB_XPASS;
  static constexpr int ypass = sizeof(T) == 4 && N == 1024 ? PS_MINB_Y1024 : sizeof(T) == 4 && N == 512 ? PS_MINB_Y512 : 0;
  static constexpr int zfwd = sizeof(T) == 4 && N == 1024 ? PS_MINB_ZF1024 : sizeof(T) == 4 && N == 512 ? PS_MINB_ZF512 : 0;
};

__device__ __forceinline__ int sidx(int n, int N) { return n < N / 2 ? n : n - N; }
__device__ __forceinline__ int rowof(int s, int wrap) { return s >= 0 ? s : s + wrap; }
__device__ __forceinline__ bool in_cube(const Geo& g, int p, int q, int r) {
  return p <= g.Kx && q <= g.Ky && q >= -g.Ky && r <= g.Kz && r >= -g.Kz;
}
// (p/(Nx/3))^2 + (q/(Ny/3))^2 + (r/(Nz/3))^2 < 1 in exact integer arithmetic
__device__ __forceinline__ bool in_sphere(const Geo& g, int p, int q, int r) {
  const long long nx2 = (long long)g.nx * g.nx, ny2 = (long long)g.ny * g.ny, nz2 = (long long)g.nz * g.nz;
  const long long lhs = 9LL * ((long long)p * p * ny2 * nz2 + (long long)q * q * nx2 * nz2 + (long long)r * r * nx2 * ny2);
  return lhs < nx2 * ny2 * nz2;
}
__device__ __forceinline__ bool kept(const Geo& g, int p, int q, int r) {
  return in_cube(g, p, q, r) && (!g.sphere || in_sphere(g, p, q, r));
}

// Loads of pass data.  COH = false: the read-only (non-coherent) path, for
// kernels that never read what they or a concurrent CTA wrote.  COH = true:
// ordinary (coherent) global loads, for data that other CTAs of the same
// launch wrote before a release/acquire handshake (the persistent ensemble
// kernel, whose passes run inside one launch: a CTA acquires the completion
// of the previous pass before it reads that pass's output).
template <bool COH = false, typename V> __device__ __forceinline__ V ldv(const V* p) {
  if constexpr (COH) return *p;
  else return __ldg(p);
}

// Sum of a per-thread double over the CTA; returns the total in thread 0.
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0;
  if (threadIdx.x == 0)
    for (int i = 0; i < nw; ++i) t += red[i];
  return t;
}

__device__ __forceinline__ double block_max(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0;
  if (threadIdx.x == 0)
    for (int i = 0; i < nw; ++i) t = fmax(t, red[i]);
  return t;
}

// ---------------------------------------------------------------------------
// zinv: curl + backward transform along z.  CTA = TX kx columns x NB retained
// ky rows.  For MHD (a.ng = 2) the velocity group (u, omega) is followed by the
// magnetic group (B, j = curl B), fields 6..11.  The CTA first copies its three input columns (retained kz rows
// only) into shared memory with cp.async, so that all its HBM reads are in
// flight at once; the six transforms then read the tile from shared memory.
// Thread (line, j0, bb) holds kz indices n = j0 + m N/E.
// ---------------------------------------------------------------------------
// Tile coordinates of a pass: the launch's block index (one kernel per pass),
// or an explicit tile of a persistent launch.  Read where the kernels read
// blockIdx, so that the per-pass kernels compile as before.
struct LaunchTile {
  __device__ __forceinline__ int x() const { return blockIdx.x; }
  __device__ __forceinline__ int y() const { return blockIdx.y; }
  __device__ __forceinline__ int z() const { return blockIdx.z; }
  __device__ __forceinline__ int gx() const { return gridDim.x; }
};
struct WorkTile {
  int bx, by, bz, ngx;
  __device__ __forceinline__ int x() const { return bx; }
  __device__ __forceinline__ int y() const { return by; }
  __device__ __forceinline__ int z() const { return bz; }
  __device__ __forceinline__ int gx() const { return ngx; }
};

// One CTA tile (x, y) of the pass; gx = tiles along x (energy partial index
// y gx + x).  COH: coherent loads (see ldv).
template <typename T, int N, int NG, int NSC, bool COH, int VAR, class TL>
__device__ __forceinline__ void zinv_tile(const PassArgs& a, const TL& tl) {
  using V = typename cplx<T>::type;
  using SH = ColShape<T, N, 0, VAR>;
  constexpr int E = SH::E, G = SH::G, TX = SH::TX, NB = SH::NB;
  constexpr int NTH = SH::NTH;
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ double red[32];
  const Geo& g = a.g;
  V* xbuf = reinterpret_cast<V*>(smraw);     // exchange: NB lines x N x TX (single buffer)
  V* tile = xbuf + NB * N * TX;              // input: [3][NB][cz][TX]
  const int tid = threadIdx.x;
  const int line = tid % TX, rest = tid / TX, j0 = rest % G, bb = rest / G;
  const int iy = tl.y() * NB + bb;
  const bool bvalid = iy < g.cy;
  const int kx = tl.x() * TX + line;  // local column
  const int kxg = g.kx0 + kx;              // its global kx
  const int q = iy <= g.Ky ? iy : iy - g.cy;
  ColumnExchange<V, ilog2<Sched<N, E>::R0>::v, 1> ex{xbuf + bb * N * TX, 0, TX, line, 0};
  const V* tw = static_cast<const V*>(a.tw_z);
  V* out = static_cast<V*>(a.a6);
  const T skx = T(kxg) * pick<T>(g.sx, g.sxf), sky = T(q) * pick<T>(g.sy, g.syf), sz = pick<T>(g.sz, g.szf);
  const long long fstride = (long long)g.nz * g.cy * g.kxp;
  const long long zstride = (long long)g.cy * g.kxp;
  const int cst = NB * g.cz * TX;                 // component stride in the tile
  const V* tb = tile + bb * g.cz * TX + line;     // this thread's column
  double esum = 0.0;
  // one group of three components at a time: u (and then B for MHD); then,
  // for the Boussinesq system, the scalar theta (one component) whose
  // gradient i k theta_hat is transformed (three fields)
#pragma unroll 1
  for (int grp = 0; grp < NG + NSC; ++grp) {
  const bool sc = grp >= NG;
  const int ncs = sc ? 1 : 3, nout = sc ? 3 : 6;
  const V* in = static_cast<const V*>(a.in.p) + 3 * grp * a.in.cs;
  // stage the tile: element (c, b, i, col) <- u_c(kx0 + col, q_b, r_i) at
  // tile[((c NB + b) cz + i) TX + col]; thread tid keeps column tid % TX and
  // walks the rows (c, b, i) with stride NTH / TX (counters, no division)
  {
    static_assert(NTH % TX == 0, "whole rows per pass");
    constexpr int RSTEP = NTH / TX;
    const int col = tid % TX;
    const int kxc = tl.x() * TX + col;
    if (kxc < ncols(g)) {
      int i = tid / TX, b = 0, c = 0;
      while (i >= g.cz) {
        i -= g.cz;
        if (++b == NB) {
          b = 0;
          ++c;
        }
      }
      V* dst = tile + (tid / TX) * TX + col;
      for (; c < ncs; dst += RSTEP * TX) {
        const int iyb = tl.y() * NB + b;
        if (iyb < g.cy) {
          const int qb = iyb <= g.Ky ? iyb : iyb - g.cy;
          const int r = i <= g.Kz ? i : i - g.cz;
          const V* src = in + c * a.in.cs + (long long)rowof(r, a.in.zwrap) * a.in.zs +
                         (long long)rowof(qb, a.in.ywrap) * a.in.ys + kxc;
          if constexpr (sizeof(V) == 8) cp_async8(dst, src);
          else cp_async16(dst, src);
        }
        i += RSTEP;
        while (i >= g.cz) {
          i -= g.cz;
          if (++b == NB) {
            b = 0;
            ++c;
          }
        }
      }
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
  }
  unsigned keepm = 0;  // bit m: mode (kx, q, r(n)) of element m is retained
#pragma unroll
  for (int m = 0; m < E; ++m)
    if (bvalid && kx < ncols(g) && kept(g, kxg, q, sidx(j0 + m * (N / E), N))) keepm |= 1u << m;
#pragma unroll 1
  for (int f = 0; f < nout; ++f) {
    V x[E];
    T ssq = 0;
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int n = j0 + m * (N / E);
      const int r = sidx(n, N);
      V v = czero<V>();
      if ((keepm >> m) & 1u) {
        const V* pm = tb + rowof(r, g.cz) * TX;
        if (sc) {
          // grad theta: i k_f theta_hat
          const V t = pm[0];
          if (f == 0) ssq += t.x * t.x + t.y * t.y;
          v = cmul_i(cscale(t, f == 0 ? skx : f == 1 ? sky : T(r) * sz));
        } else if (f < 3) {
          v = pm[f * cst];
          ssq += v.x * v.x + v.y * v.y;
        } else {
          const T skz = T(r) * sz;
          // omega_hat = i k x u_hat
          if (f == 3) {
            const V uy = pm[cst], uz = pm[2 * cst];
            v = cmul_i(csub(cscale(uz, sky), cscale(uy, skz)));
          } else if (f == 4) {
            const V ux = pm[0], uz = pm[2 * cst];
            v = cmul_i(csub(cscale(ux, skz), cscale(uz, skx)));
          } else {
            const V ux = pm[0], uy = pm[cst];
            v = cmul_i(csub(cscale(uy, skx), cscale(ux, sky)));
          }
        }
      }
      x[m] = v;
    }
    if (a.e_part && f < 3) esum += (double)ssq;
    line_fft<N, E, +1>(x, j0, tw, ex);
    if (bvalid) {
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const int n = j0 + m * (N / E);
        out[(6 * grp + f) * fstride + n * zstride + (long long)iy * g.kxp + kx] = x[m];
      }
    }
  }
  __syncthreads();  // the tile is restaged for the next group
  }
  if (a.e_part) {
    // energy 1/2 sum w |u|^2 (+ |B|^2 or theta^2), w = 1 on the kx = 0 plane, else 2
    const double t = block_sum(esum * (kxg == 0 ? 0.5 : 1.0), red);
    if (threadIdx.x == 0) a.e_part[tl.y() * tl.gx() + tl.x()] = t;
  }
}

template <typename T, int N, int NG, int NSC, int VAR = 0>
__global__ void __launch_bounds__(ColShape<T, N, 0, VAR>::NTH, MinB<T, N>::zinv) k_zinv(const PassArgs a) {
  zinv_tile<T, N, NG, NSC, false, VAR>(a, LaunchTile{});
}

// ---------------------------------------------------------------------------
// yinv: backward transform along y of 6 fields.  CTA = TX columns x NB z planes.
// ---------------------------------------------------------------------------
template <typename T, int N, bool COH, int VAR, class TL>
__device__ __forceinline__ void yinv_tile(const PassArgs& a, const TL& tl) {
  using V = typename cplx<T>::type;
  using SH = ColShape<T, N, 1, VAR>;
  constexpr int E = SH::E, G = SH::G, TX = SH::TX, NB = SH::NB;
  extern __shared__ __align__(128) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const Geo& g = a.g;
  const int tid = threadIdx.x;
  const int line = tid % TX, rest = tid / TX, j0 = rest % G, bb = rest / G;
  const int iz = tl.y() * NB + bb;
  const bool bvalid = iz < g.nz;
  const int kx = tl.x() * TX + line;
  const int f = tl.z();
  ColumnExchange<V, ilog2<Sched<N, E>::R0>::v, ColBuf<T, N>::v> ex{sm + bb * N * TX, NB * N * TX, TX, line, 0};
  const V* in = static_cast<const V*>(a.a6) + ((long long)f * g.nz + (bvalid ? iz : 0)) * g.cy * g.kxp + kx;
  V* out = static_cast<V*>(a.b6) + ((long long)f * g.nz + (bvalid ? iz : 0)) * g.ny * g.kxp + kx;
  V x[E];
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int n = j0 + m * (N / E);
    const int q = sidx(n, N);
    V v = czero<V>();
    if (bvalid && q <= g.Ky && q >= -g.Ky) v = ldv<COH>(in + (long long)rowof(q, g.cy) * g.kxp);
    x[m] = v;
  }
  line_fft<N, E, +1>(x, j0, static_cast<const V*>(a.tw_y), ex);
  if (bvalid) {
#pragma unroll
    for (int m = 0; m < E; ++m) out[(long long)(j0 + m * (N / E)) * g.kxp] = x[m];
  }
}

template <typename T, int N, int VAR = 0>
__global__ void __launch_bounds__(ColShape<T, N, 1, VAR>::NTH, MinB<T, N>::ypass) k_yinv(const PassArgs a) {
  yinv_tile<T, N, false, VAR>(a, LaunchTile{});
}

// ---------------------------------------------------------------------------
// xpass: per physical (z, y) row.  Persistent CTAs loop over groups of rpc
// consecutive rows.  The input rows of a group are brought into shared memory
// by TMA bulk copies; once every thread has gathered its points into registers
// the copies of the next group are issued into the same stage, so they land
// while the current group is transformed.  Thread j0 of a row's group of G
// threads holds the points n = j0 + m N/E.  The packed lines of a row are
// transformed together (line_fft_rows): the inverse lines three at a time, the
// forward lines of the products together, one exchange for all of them.
// NG = 2 (MHD): u + i omega and B + i j in, u x omega + j x B and u x B out.
// NSC = 1 (Boussinesq): u + i omega and grad theta in, u x omega and
// u . grad theta out.
// ---------------------------------------------------------------------------
// The work of the x pass on one row: gather the packed inverse lines (field f
// of the row at st + f fst, retained kx only), transform them, form the
// products, transform forward, split and store the retained kx of the output
// row.  `gathered` runs once every thread holds its points (the TMA kernel
// refills its stage there).  COH: st is global memory written earlier in the
// same launch (coherent loads).
// XE: points per thread (the x pass's schedule unless a caller picks another).
template <typename T, int N, int NG, int NSC, bool COH, class TW, class AfterGather, int XE = EPass<T, N, 3>::v>
__device__ __forceinline__ void xpass_row(const PassArgs& a, const long long row, const bool rvalid, const int j0,
                                          const typename cplx<T>::type* st, const long long fst, const TW& tw,
                                          LinesExchange<typename cplx<T>::type, 1>& ex, T& umax2,
                                          AfterGather&& gathered) {
  using V = typename cplx<T>::type;
  constexpr int E = XE;
  constexpr int NLI = 3 * NG + 2 * NSC;  // inverse packed lines
  constexpr bool HD = NG == 1 && NSC == 0;
  constexpr int NFW = NG == 2 ? 3 : 2;  // forward packed lines
  const Geo& g = a.g;
  const int kxp = g.kxp;
  const long long rows = (long long)g.nz * g.ny;
  V* C = static_cast<V*>(a.a6);
  // packed lines: u_c + i omega_c (c < 3) and, for MHD, B_c + i j_c; for
  // the Boussinesq system d_x theta + i d_y theta and d_z theta + i 0
  V U[NLI][E];
#pragma unroll
  for (int c = 0; c < NLI; ++c) {
    const bool scl = NSC && c == 4;  // the unpaired line
    // real and imaginary part fields
    const int fr = c < 3 ? c : NSC ? (c == 3 ? 6 : 8) : 6 + (c - 3);
    const int fi = c < 3 ? c + 3 : NSC ? (c == 3 ? 7 : 8) : 9 + (c - 3);
    const V* pu = st + fr * fst;
    const V* pw = st + fi * fst;
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int n = j0 + m * (N / E);
      // full spectrum C[n] = a_hat[n] + i b_hat[n]; for n > N/2 the entries
      // are conj(a_hat[N-n]) + i conj(b_hat[N-n]) (real a and b)
      const bool hi = n > N / 2;
      const int p = hi ? N - n : n;
      V v = czero<V>();
      if (rvalid && p <= g.Kx) {
        V X, W;
        if constexpr (COH) {
          X = ldv<true>(pu + p);
          W = ldv<true>(pw + p);
        } else {
          X = pu[p];
          W = pw[p];
        }
        if (hi) {
          X = cconj(X);
          W = cconj(W);
        }
        v = scl ? X : mk<V>(X.x - W.y, X.y + W.x);
      }
      U[c][m] = v;
    }
  }
  gathered();
  if constexpr (HD) {
    line_fft_rows<N, E, +1>(U, j0, tw, ex);
  } else if constexpr (NSC == 1) {
    V L[3][E], S[2][E];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int m = 0; m < E; ++m) L[c][m] = U[c][m];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int m = 0; m < E; ++m) S[c][m] = U[3 + c][m];
    line_fft_rows<N, E, +1>(L, j0, tw, ex);
    line_fft_rows<N, E, +1>(S, j0, tw, ex);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int m = 0; m < E; ++m) U[c][m] = L[c][m];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int m = 0; m < E; ++m) U[3 + c][m] = S[c][m];
  } else {
#pragma unroll
    for (int h = 0; h < NG; ++h) {
      V L[3][E];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int m = 0; m < E; ++m) L[c][m] = U[3 * h + c][m];
      line_fft_rows<N, E, +1>(L, j0, tw, ex);
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int m = 0; m < E; ++m) U[3 * h + c][m] = L[c][m];
    }
  }
  // products at the thread's points (real part = field, imaginary = curl)
  V F[NFW][E];
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const T ux = U[0][m].x, uy = U[1][m].x, uz = U[2][m].x;
    const T wx = U[0][m].y, wy = U[1][m].y, wz = U[2][m].y;
    umax2 = fmax(umax2, ux * ux + uy * uy + uz * uz);
    T nx = uy * wz - uz * wy, ny = uz * wx - ux * wz, nz = ux * wy - uy * wx;
    if constexpr (HD) {
      F[0][m] = mk<V>(nx, ny);
      F[1][m] = mk<V>(nz, T(0));
    } else if constexpr (NSC == 1) {
      // u . grad theta
      const T adv = ux * U[3][m].x + uy * U[3][m].y + uz * U[4][m].x;
      F[0][m] = mk<V>(nx, ny);
      F[1][m] = mk<V>(nz, adv);
    } else {
      const T bx = U[3][m].x, by = U[4][m].x, bz = U[5][m].x;
      const T jx = U[3][m].y, jy = U[4][m].y, jz = U[5][m].y;
      nx += jy * bz - jz * by;  // + j x B
      ny += jz * bx - jx * bz;
      nz += jx * by - jy * bx;
      const T ex_ = uy * bz - uz * by, ey_ = uz * bx - ux * bz, ez_ = ux * by - uy * bx;  // u x B
      F[0][m] = mk<V>(nx, ny);
      F[1][m] = mk<V>(nz, ex_);
      F[2][m] = mk<V>(ey_, ez_);
    }
  }
  if (!a.xdiag) {  // uniform across the grid
    line_fft_rows<N, E, -1>(F, j0, tw, ex);
    const long long rrow = rvalid ? row : 0;
    const int kend = kxp < N / 2 + 1 ? kxp : N / 2 + 1;
    // split each packed transform F = DFT(a) + i DFT(b) of two real fields
    // with its mirrored entry F[N-k] (all split lines through one exchange);
    // for HD the second line has b = 0
    constexpr int NSP = HD ? 1 : NFW;  // lines that need the split
#pragma unroll
    for (int w = 0; w < NSP; ++w)
#pragma unroll
      for (int m = 0; m < E; ++m) ex.template put<0, 0>(w, j0 + m * (N / E), F[w][m]);
    ex.sync();
#pragma unroll
    for (int w = 0; w < NFW; ++w) {
      const bool split = w < NSP;
      V* ca = C + ((long long)(2 * w) * rows + rrow) * kxp;
      V* cb = C + ((long long)(2 * w + 1) * rows + rrow) * kxp;
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const int k = j0 + m * (N / E);
        if (rvalid && k < kend) {
          V va = czero<V>(), vb = czero<V>();
          if (k <= g.Kx) {
            const V Fk = F[w][m];
            if (split) {
              const V Fm = cconj(ex.template get<0, 0>(w, k == 0 ? 0 : N - k));
              va = cscale(cadd(Fk, Fm), T(0.5));
              vb = cscale(cmul_mi(csub(Fk, Fm)), T(0.5));
            } else {
              va = Fk;
            }
          }
          ca[k] = va;
          if (split) cb[k] = vb;
        }
      }
    }
  }
}

template <typename T, int N, int NG, int NSC>
__global__ void __launch_bounds__(RPCOf<T, N>::v * (N / EPass<T, N, 3>::v),
                                  NG == 1 && NSC == 0 ? MinB<T, N>::xpass : 1)
    k_xpass(const PassArgs a, const int rpc) {
  using V = typename cplx<T>::type;
  constexpr int E = EPass<T, N, 3>::v, G = N / E;
  constexpr int NF = 6 * NG + 3 * NSC;  // input fields: u, omega (, B, j) (, grad theta)
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ double red[32];
  __shared__ __align__(8) uint64_t bar[1];
  __shared__ int abort_flag;
  const Geo& g = a.g;
  const int kxp = g.kxp;
  const int tid = threadIdx.x;
  const int j0 = tid % G, rl = tid / G;
  const long long rows = (long long)g.nz * g.ny;
  const long long ngroups = (rows + rpc - 1) / rpc;
  V* stage = reinterpret_cast<V*>(smraw);
  V* exbuf = stage + NF * rpc * kxp;
  // exchange region of this row: XLINES lines of N slots, single buffer
  LinesExchange<V, 1> ex{exbuf + rl * XLINES * N, N, 0, 0};
  // rows are independent between the group barriers: sync only the row's threads
  if (G >= 32) {
    ex.bar_id = 1 + rl;
    ex.nthr = G;
  } else {
    ex.bar_id = -1;
  }
  // stage twiddles: in registers when few, else a per-thread table in shared
  // memory (thread j0 of every row reads its own column), else global memory
  constexpr bool TR = XTwReg<T, N>::v;
  constexpr bool TT = !TR && XTwTable<T, N>::v;
  using TwAcc = typename std::conditional<TR, RegTw<V, N, E>,
                typename std::conditional<TT, ThreadTw<V, N, E>, GlobalTw<V>>::type>::type;
  TwAcc tw;
  if constexpr (TR) {
    tw.load(static_cast<const V*>(a.tw_x), j0);
  } else if constexpr (TT) {
    V* twt = exbuf + rpc * XLINES * N;
    if (rl == 0) fill_thread_tw<N, E>(twt, static_cast<const V*>(a.tw_x), j0);
    tw = TwAcc{twt, j0};
  } else {
    tw = TwAcc{static_cast<const V*>(a.tw_x)};
  }
  const V* B = static_cast<const V*>(a.b6);
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    abort_flag = 0;
    mbar_fence_init();
  }
  __syncthreads();
  // stage <- the NF input fields of row group grp (rpc contiguous rows each)
  auto issue = [&](long long grp) {
    const long long r0 = grp * rpc;
    const long long nr = rows - r0 < rpc ? rows - r0 : rpc;
    const uint32_t bytes = (uint32_t)(nr * kxp * sizeof(V));
    mbar_arrive_expect_tx(&bar[0], (uint32_t)NF * bytes);
    for (int c = 0; c < NF; ++c)
      bulk_g2s(stage + c * rpc * kxp, B + ((long long)c * rows + r0) * kxp, bytes, &bar[0]);
  };
  uint32_t ph = 0u;  // completed-phase parity of the stage barrier
  long long it = blockIdx.x;
  const uint32_t polls = a.wait_polls ? a.wait_polls : PS_WAIT_LIMIT;
  // thread 0: a copy into the stage is in flight (the test hook never issues
  // the first one, so that the wait below runs out)
  bool inflight = false;
  if (tid == 0 && it < ngroups && !a.wait_test) {
    issue(it);
    inflight = true;
  }
  T umax2 = 0;
  while (it < ngroups) {
    const long long nxt = it + gridDim.x;
    const uint32_t cur = ph;
    ph ^= 1u;
    if (!mbar_wait(&bar[0], cur, polls)) abort_flag = 1;
    __syncthreads();
    if (abort_flag) {
      if (tid == 0) {
        atomicExch(a.err, PS_DEV_TIMEOUT_XPASS);
        // bounded: let a copy still in flight land before the CTA exits
        if (inflight) mbar_wait(&bar[0], cur, PS_DRAIN_LIMIT);
      }
      break;
    }
    const long long row = it * rpc + rl;
    xpass_row<T, N, NG, NSC, false>(a, row, row < rows, j0, stage + rl * kxp, (long long)rpc * kxp, tw, ex, umax2,
                                   [&] {
                                     // every thread has its points: the stage takes the next group's rows
                                     __syncthreads();
                                     if (tid == 0) {
                                       inflight = nxt < ngroups;
                                       if (inflight) {
                                         fence_proxy_async();
                                         issue(nxt);
                                       }
                                     }
                                   });
    __syncthreads();  // the exchange buffers are free again
    it = nxt;
  }
  if (a.umax2) {
    const double t = block_max((double)umax2, red);
    if (threadIdx.x == 0) atomicMax(a.umax2, (unsigned long long)__double_as_longlong(t));
  }
}

// ---------------------------------------------------------------------------
// yfwd: forward transform along y of 3 fields, keep |ky| <= Ky.
// ---------------------------------------------------------------------------
template <typename T, int N, bool COH, int VAR, class TL>
__device__ __forceinline__ void yfwd_tile(const PassArgs& a, const TL& tl) {
  using V = typename cplx<T>::type;
  using SH = ColShape<T, N, 1, VAR>;
  constexpr int E = SH::E, G = SH::G, TX = SH::TX, NB = SH::NB;
  extern __shared__ __align__(128) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const Geo& g = a.g;
  const int tid = threadIdx.x;
  const int line = tid % TX, rest = tid / TX, j0 = rest % G, bb = rest / G;
  const int iz = tl.y() * NB + bb;
  const bool bvalid = iz < g.nz;
  const int kx = tl.x() * TX + line;
  const int f = tl.z();
  ColumnExchange<V, ilog2<Sched<N, E>::R0>::v, ColBuf<T, N>::v> ex{sm + bb * N * TX, NB * N * TX, TX, line, 0};
  const V* in = static_cast<const V*>(a.a6) + ((long long)f * g.nz + (bvalid ? iz : 0)) * g.ny * g.kxp + kx;
  V* out = static_cast<V*>(a.b6) + ((long long)f * g.nz + (bvalid ? iz : 0)) * g.cy * g.kxp + kx;
  V x[E];
#pragma unroll
  for (int m = 0; m < E; ++m) x[m] = bvalid ? ldv<COH>(in + (long long)(j0 + m * (N / E)) * g.kxp) : czero<V>();
  line_fft<N, E, -1>(x, j0, static_cast<const V*>(a.tw_y), ex);
  if (bvalid) {
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int q = sidx(j0 + m * (N / E), N);
      if (q <= g.Ky && q >= -g.Ky) out[(long long)rowof(q, g.cy) * g.kxp] = x[m];
    }
  }
}

template <typename T, int N, int VAR = 0>
__global__ void __launch_bounds__(ColShape<T, N, 1, VAR>::NTH, MinB<T, N>::ypass) k_yfwd(const PassArgs a) {
  yfwd_tile<T, N, false, VAR>(a, LaunchTile{});
}

// ---------------------------------------------------------------------------
// zfwd: forward transform along z of one field per CTA (blockIdx.z), keep the
// retained kz rows and scale by 1/(Nx Ny Nz).  Writes the compact transformed
// nonlinear term [3 ng][cz][cy][kxp] into a6 (zero where the mode is not
// retained).  The projection, forcing and stage update follow in k_update.
// ---------------------------------------------------------------------------
template <typename T, int N, bool COH, int VAR, class TL>
__device__ __forceinline__ void zfwd_tile(const PassArgs& a, const TL& tl) {
  using V = typename cplx<T>::type;
  using SH = ColShape<T, N, 2, VAR>;
  constexpr int E = SH::E, G = SH::G, TX = SH::TX, NB = SH::NB;
  extern __shared__ __align__(128) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  const Geo& g = a.g;
  const int tid = threadIdx.x;
  const int line = tid % TX, rest = tid / TX, j0 = rest % G, bb = rest / G;
  const int iy = tl.y() * NB + bb;
  const bool bvalid = iy < g.cy;
  const int kx = tl.x() * TX + line;
  const int q = iy <= g.Ky ? iy : iy - g.cy;
  const int f = tl.z();
  ColumnExchange<V, ilog2<Sched<N, E>::R0>::v, ColBuf<T, N>::v> ex{sm + bb * N * TX, NB * N * TX, TX, line, 0};
  const long long cs_in = (long long)g.nz * g.cy * g.kxp;
  const V* in = static_cast<const V*>(a.b6) + f * cs_in + (long long)(bvalid ? iy : 0) * g.kxp + kx;
  V x[E];
#pragma unroll
  for (int m = 0; m < E; ++m)
    x[m] = bvalid ? ldv<COH>(in + (long long)(j0 + m * (N / E)) * g.cy * g.kxp) : czero<V>();
  line_fft<N, E, -1>(x, j0, static_cast<const V*>(a.tw_z), ex);
  if (bvalid) {
    const T inv = pick<T>(a.inv_n3, a.inv_n3f);
    V* out = static_cast<V*>(a.a6) + (long long)f * g.cz * g.cy * g.kxp + (long long)iy * g.kxp + kx;
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int r = sidx(j0 + m * (N / E), N);
      if (r <= g.Kz && r >= -g.Kz)
        out[(long long)rowof(r, g.cz) * g.cy * g.kxp] =
            kx < ncols(g) && kept(g, g.kx0 + kx, q, r) ? cscale(x[m], inv) : czero<V>();
    }
  }
}

template <typename T, int N, int VAR = 0>
__global__ void __launch_bounds__(ColShape<T, N, 2, VAR>::NTH, MinB<T, N>::zfwd) k_zfwd(const PassArgs a) {
  zfwd_tile<T, N, false, VAR>(a, LaunchTile{});
}

// ---------------------------------------------------------------------------
// update: per mode, from the compact transformed nonlinear term Nh (a6)
//   velocity group: v = P(Nh + f + closure - n_bv theta z), P = I - k k^T/|k|^2,
//                   v(0) = 0 (the buoyancy term only for the Boussinesq system)
//   magnetic group: v = i k x Nh  (the curl of u x B)
//   scalar:         v = -Nh(u . grad theta) + n_bv w  (Boussinesq)
// with theta and w of the stage input; then the selected output (ZfwdMode):
// the right-hand side v - damp |k|^2 u, or a Lawson RK stage update of the
// compact stage buffers / the caller's state.
// full != 0: one thread per mode of the caller's layout (modes outside the
// retained set are written as zero); otherwise one thread per retained mode.
// Consecutive threads take consecutive kx: every access is a contiguous row.
// ---------------------------------------------------------------------------
template <typename T, int NG, int NSC, bool SLAB, bool COH>
__device__ __forceinline__ void update_mode(const PassArgs& a, const int full, const unsigned idx) {
  using V = typename cplx<T>::type;
  constexpr int NC = 3 * NG + NSC;  // state components
  const Geo& g = a.g;
  // a whole problem (not a kx slab) has rows of nh entries and cx columns
  const unsigned rl = SLAB ? rowlen(g) : g.nh, nc = SLAB ? ncols(g) : g.cx;
  int kx, q, r;  // kx: local column (array index); kxg = g.kx0 + kx its global kx
  long long orow = 0;  // row of the caller layout (z * ny + y)
  if (full) {
    if (idx >= (unsigned)g.nz * (unsigned)g.ny * rl) return;
    kx = (int)(idx % rl);
    const unsigned orow32 = idx / rl;
    orow = orow32;
    q = sidx((int)(orow32 % (unsigned)g.ny), g.ny);
    r = sidx((int)(orow32 / (unsigned)g.ny), g.nz);
  } else {
    if (idx >= (unsigned)g.cz * (unsigned)g.cy * nc) return;
    kx = (int)(idx % nc);
    const unsigned crow = idx / nc;
    const int iy = (int)(crow % (unsigned)g.cy), iz = (int)(crow / (unsigned)g.cy);
    q = iy <= g.Ky ? iy : iy - g.cy;
    r = iz <= g.Kz ? iz : iz - g.cz;
  }
  const int kxg = SLAB ? g.kx0 + kx : kx;
  const long long fcs = (long long)g.nz * g.ny * rl;  // caller layout component stride
  const bool keep = (!SLAB || kx < nc) && kept(g, kxg, q, r);
  if (!keep) {
    if (full) {
      V* po = static_cast<V*>(a.out_full) + orow * rl + kx;
#pragma unroll
      for (int c = 0; c < NC; ++c) po[c * fcs] = czero<V>();
    }
    return;
  }
  // a bounded wait of this right-hand side gave up: its nonlinear term is
  // incomplete, so every retained output becomes NaN instead of a wrong value
  const bool failed = *a.err != 0;
  const int iy = rowof(q, g.cy), iz = rowof(r, g.cz);
  const long long ccs = (long long)g.cz * g.cy * g.kxp;  // compact component stride
  const long long ci = ((long long)iz * g.cy + iy) * g.kxp + kx;
  const T kxv = T(kxg) * pick<T>(g.sx, g.sxf), kyv = T(q) * pick<T>(g.sy, g.syf), kzv = T(r) * pick<T>(g.sz, g.szf);
  const T k2 = kxv * kxv + kyv * kyv + kzv * kzv;
  const T dt = pick<T>(a.dt, a.dtf);
  const V* nh = static_cast<const V*>(a.a6);
  V w_s = czero<V>(), th_s = czero<V>();  // Boussinesq: w and theta of the stage input
  if constexpr (NSC == 1) {
    const V* pi = static_cast<const V*>(a.in.p) + (long long)rowof(r, a.in.zwrap) * a.in.zs +
                  (long long)rowof(q, a.in.ywrap) * a.in.ys + kx;
    w_s = ldv<COH>(pi + 2 * a.in.cs);
    th_s = ldv<COH>(pi + 3 * a.in.cs);
  }
#pragma unroll
  for (int grp = 0; grp < NG + NSC; ++grp) {
    const bool scl = NSC == 1 && grp == NG;  // the scalar (one component)
    const bool mag = NG == 2 && grp == 1;
    const int c0 = 3 * grp;
    const int nc = scl ? 1 : 3;
    V kk[3];
    if (scl) {
      kk[0] = csub(cscale(w_s, pick<T>(a.n_bv, a.nbvf)), ldv<COH>(nh + 3 * ccs + ci));
      kk[1] = kk[2] = czero<V>();
    } else {
      V v0 = ldv<COH>(nh + (c0 + 0) * ccs + ci), v1 = ldv<COH>(nh + (c0 + 1) * ccs + ci), v2 = ldv<COH>(nh + (c0 + 2) * ccs + ci);
      if (!mag) {
        if (a.extra) {  // closure term (LES), compact layout
          const V* ex0 = static_cast<const V*>(a.extra) + ci;
          v0 = cadd(v0, ldv<COH>(ex0));
          v1 = cadd(v1, ldv<COH>(ex0 + ccs));
          v2 = cadd(v2, ldv<COH>(ex0 + 2 * ccs));
        }
        const V* fb = static_cast<const V*>(a.fbox);
        if (fb && kx <= a.Fx && q <= a.Fy && q >= -a.Fy && r <= a.Fz && r >= -a.Fz) {
          const long long fzs = (long long)(2 * a.Fy + 1) * (a.Fx + 1);
          const long long fcs2 = (long long)(2 * a.Fz + 1) * fzs;
          const long long fo = (long long)(r + a.Fz) * fzs + (long long)(q + a.Fy) * (a.Fx + 1) + kx;
          v0 = cadd(v0, ldv<COH>(fb + fo));
          v1 = cadd(v1, ldv<COH>(fb + fo + fcs2));
          v2 = cadd(v2, ldv<COH>(fb + fo + 2 * fcs2));
        }
        if constexpr (NSC == 1) v2 = csub(v2, cscale(th_s, pick<T>(a.n_bv, a.nbvf)));  // buoyancy -N theta z
        if (k2 > T(0)) {
          // Leray projection v - k (k.v)/|k|^2
          const V kd = cadd(cadd(cscale(v0, kxv), cscale(v1, kyv)), cscale(v2, kzv));
          const T ik2 = T(1) / k2;
          v0 = csub(v0, cscale(kd, kxv * ik2));
          v1 = csub(v1, cscale(kd, kyv * ik2));
          v2 = csub(v2, cscale(kd, kzv * ik2));
        } else {
          v0 = v1 = v2 = czero<V>();
        }
      } else {
        // curl(u x B): i k x v
        const V w0 = cmul_i(csub(cscale(v2, kyv), cscale(v1, kzv)));
        const V w1 = cmul_i(csub(cscale(v0, kzv), cscale(v2, kxv)));
        const V w2 = cmul_i(csub(cscale(v1, kxv), cscale(v0, kyv)));
        v0 = w0;
        v1 = w1;
        v2 = w2;
      }
      kk[0] = v0;
      kk[1] = v1;
      kk[2] = v2;
    }
    if (failed) {
      const T qnan = T(NAN);
      kk[0] = kk[1] = kk[2] = mk<V>(qnan, qnan);
    }
    const V* pu = static_cast<const V*>(a.u_n.p) + c0 * a.u_n.cs + (long long)rowof(r, a.u_n.zwrap) * a.u_n.zs +
                  (long long)rowof(q, a.u_n.ywrap) * a.u_n.ys + kx;
    V* po = static_cast<V*>(a.out_full) + c0 * fcs + orow * rl + kx;
    const bool second = mag || scl;  // diffusivity and factor tables of the second field
    if (a.mode == ZF_RHS) {
      const T vk = (second ? pick<T>(a.eta, a.etaf) : pick<T>(a.nu, a.nuf)) * k2;
#pragma unroll
      for (int c = 0; c < nc; ++c) po[c * fcs] = csub(kk[c], cscale(ldv<COH>(pu + c * a.u_n.cs), vk));
      continue;
    }
    // Lawson RK with E = exp(-damp |k|^2 dt/2) = ex(p) ey(q) ez(r)
    const T* ifx = static_cast<const T*>(second ? a.jfx : a.ifx);
    const T* ify = static_cast<const T*>(second ? a.jfy : a.ify);
    const T* ifz = static_cast<const T*>(second ? a.jfz : a.ifz);
    const T Ef = __ldg(ifx + kxg) * __ldg(ify + iy) * __ldg(ifz + iz);
    const T E2 = Ef * Ef;
    V* acc = static_cast<V*>(a.acc) + c0 * ccs + ci;
    V* nxt = static_cast<V*>(a.nxt) + c0 * ccs + ci;
    V u[3], ac[3];
#pragma unroll
    for (int c = 0; c < nc; ++c) {
      u[c] = ldv<COH>(pu + c * a.u_n.cs);
      ac[c] = (a.mode == ZF_RK4_1 || a.mode == ZF_RK2_1) ? czero<V>() : acc[c * ccs];
    }
#pragma unroll
    for (int c = 0; c < nc; ++c) {
      const V k = kk[c];
      switch (a.mode) {
        case ZF_RK4_1:  // acc = E^2 k1 ; next = E (u + dt/2 k1)
          acc[c * ccs] = cscale(k, E2);
          nxt[c * ccs] = cscale(cadd(u[c], cscale(k, T(0.5) * dt)), Ef);
          break;
        case ZF_RK4_2:  // acc += 2 E k2 ; next = E u + dt/2 k2
          acc[c * ccs] = cadd(ac[c], cscale(k, T(2) * Ef));
          nxt[c * ccs] = cadd(cscale(u[c], Ef), cscale(k, T(0.5) * dt));
          break;
        case ZF_RK4_3:  // acc += 2 E k3 ; next = E^2 u + dt E k3
          acc[c * ccs] = cadd(ac[c], cscale(k, T(2) * Ef));
          nxt[c * ccs] = cadd(cscale(u[c], E2), cscale(k, dt * Ef));
          break;
        case ZF_RK4_4:  // u+ = E^2 u + dt/6 (acc + k4)
          po[c * fcs] = cadd(cscale(u[c], E2), cscale(cadd(ac[c], k), dt / T(6)));
          break;
        case ZF_RK2_1:  // next = E^2 (u + dt k1) ; acc = E^2 (u + dt/2 k1)
          nxt[c * ccs] = cscale(cadd(u[c], cscale(k, dt)), E2);
          acc[c * ccs] = cscale(cadd(u[c], cscale(k, T(0.5) * dt)), E2);
          break;
        case ZF_RK2_2:  // u+ = acc + dt/2 k2
          po[c * fcs] = cadd(ac[c], cscale(k, T(0.5) * dt));
          break;
        default:
          break;
      }
    }
  }
}

// 32-bit mode index (the launcher checks that the modes fit): 64-bit integer
// division runs on the FP64 pipe, which is slow on this GPU
template <typename T, int NG, int NSC, bool SLAB = false>
__global__ void __launch_bounds__(256) k_update(const PassArgs a, const int full) {
  update_mode<T, NG, NSC, SLAB, false>(a, full, blockIdx.x * blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename K>
static cudaError_t prep(K kernel, size_t smem) {
  // the 48 KB default covers static and dynamic shared memory together: opt
  // in well before the dynamic part alone reaches it
  if (smem > 32 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

// Energy partials (CTAs) of the z-inverse pass in shape VAR.
template <typename T, int N, int VAR = 0>
int zinv_grid_blocks(const Geo& g) {
  using SH = ColShape<T, N, 0, VAR>;
  return (g.kxp / SH::TX) * ((g.cy + SH::NB - 1) / SH::NB);
}

template <typename T, int N, int NG, int NSC, int VAR = 0>
cudaError_t zinv_ng(const PassArgs& a0, cudaStream_t s, int* nb) {
  PassArgs a = a0;
  prepare_args(a);
  using V = typename cplx<T>::type;
  using SH = ColShape<T, N, 0, VAR>;
  constexpr int TX = SH::TX, NB = SH::NB;
  const size_t smem = (1ull * NB * N * TX + 3ull * NB * a.g.cz * TX) * sizeof(V);
  cudaError_t e = prep(k_zinv<T, N, NG, NSC, VAR>, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.g.kxp / TX, (a.g.cy + NB - 1) / NB);
  if (nb) *nb = grid.x * grid.y;
  k_zinv<T, N, NG, NSC, VAR><<<grid, SH::NTH, smem, s>>>(a);
  return cudaGetLastError();
}
template <typename T, int N>
cudaError_t zinv_n(const PassArgs& a, cudaStream_t s, int* nb) {
  if (a.ng == 2) return zinv_ng<T, N, 2, 0>(a, s, nb);
  if (a.nsc) return zinv_ng<T, N, 1, 1>(a, s, nb);
  if constexpr (HasShapes<T, N>::v) {
    if (a.shape[0] == 1) return zinv_ng<T, N, 1, 0, 1>(a, s, nb);
    if constexpr (AltE<T, N>::v != EOf<T, N>::v)
      if (a.shape[0] == 2) return zinv_ng<T, N, 1, 0, 2>(a, s, nb);
  }
  return zinv_ng<T, N, 1, 0>(a, s, nb);
}
template <typename T, int N, int VAR = 0>
cudaError_t yinv_nv(const PassArgs& a0, cudaStream_t s) {
  PassArgs a = a0;
  prepare_args(a);
  using V = typename cplx<T>::type;
  using SH = ColShape<T, N, 1, VAR>;
  constexpr int TX = SH::TX, NB = SH::NB;
  const size_t smem = (size_t)ColBuf<T, N>::v * NB * N * TX * sizeof(V);
  cudaError_t e = prep(k_yinv<T, N, VAR>, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.g.kxp / TX, (a.g.nz + NB - 1) / NB, a.nfi);
  k_yinv<T, N, VAR><<<grid, SH::NTH, smem, s>>>(a);
  return cudaGetLastError();
}
// Shape variant v (0, 1, 2) of pass launcher L for a length with variants.
#define PS_SHAPE_DISPATCH(L, var_, ...)                                                 \
  do {                                                                                  \
    if constexpr (HasShapes<T, N>::v) {                                                 \
      if ((var_) == 1) return L<T, N, 1>(__VA_ARGS__);                                  \
      if constexpr (AltE<T, N>::v != EOf<T, N>::v)                                      \
        if ((var_) == 2) return L<T, N, 2>(__VA_ARGS__);                                \
    }                                                                                   \
    return L<T, N, 0>(__VA_ARGS__);                                                     \
  } while (0)
template <typename T, int N>
cudaError_t yinv_n(const PassArgs& a, cudaStream_t s) {
  PS_SHAPE_DISPATCH(yinv_nv, a.shape[1], a, s);
}
// Shared memory of the x pass for rpc rows: one input stage of 6 ng rows, the
// exchange region (XLINES lines per row) and, when used, the twiddle table.
template <typename T, int N>
size_t xpass_smem(const Geo& g, int rpc, int nf) {
  using V = typename cplx<T>::type;
  constexpr int E = EPass<T, N, 3>::v;
  const size_t tt = (!XTwReg<T, N>::v && XTwTable<T, N>::v) ? (size_t)TwSlots<N, E>::total * (N / E) : 0;
  return ((size_t)nf * rpc * g.kxp + (size_t)XLINES * rpc * N + tt) * sizeof(V);
}

template <typename T, int N, int NG, int NSC>
cudaError_t xpass_ng(const PassArgs& a0, cudaStream_t s) {
  PassArgs a = a0;
  prepare_args(a);
  constexpr int NF = 6 * NG + 3 * NSC;
  constexpr int E = EPass<T, N, 3>::v, G = N / E;
  // rows per CTA: as many as the launch bound allows while two CTAs fit an SM
  int rpc = RPCOf<T, N>::v;
  while (rpc > 1 && xpass_smem<T, N>(a.g, rpc, NF) > 113 * 1024) rpc /= 2;
  if (a.xrpc > 0 && a.xrpc < rpc) rpc = a.xrpc;  // tuned (smaller) row groups
  const size_t smem = xpass_smem<T, N>(a.g, rpc, NF);
  cudaError_t e = cudaFuncSetAttribute(k_xpass<T, N, NG, NSC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_xpass<T, N, NG, NSC>, rpc * G, smem)) !=
      cudaSuccess)
    return e;
  const long long rows = (long long)a.g.nz * a.g.ny;
  const long long groups = (rows + rpc - 1) / rpc;
  long long grid = (long long)nsm * (per_sm > 0 ? per_sm : 1);
  if (grid > groups) grid = groups;
  k_xpass<T, N, NG, NSC><<<(unsigned)grid, rpc * G, smem, s>>>(a, rpc);
  return cudaGetLastError();
}

template <typename T, int N>
cudaError_t xpass_n(const PassArgs& a, cudaStream_t s) {
  if (a.ng == 2) return xpass_ng<T, N, 2, 0>(a, s);
  return a.nsc ? xpass_ng<T, N, 1, 1>(a, s) : xpass_ng<T, N, 1, 0>(a, s);
}

template <typename T, int N, int VAR = 0>
cudaError_t yfwd_nv(const PassArgs& a0, cudaStream_t s) {
  PassArgs a = a0;
  prepare_args(a);
  using V = typename cplx<T>::type;
  using SH = ColShape<T, N, 1, VAR>;
  constexpr int TX = SH::TX, NB = SH::NB;
  const size_t smem = (size_t)ColBuf<T, N>::v * NB * N * TX * sizeof(V);
  cudaError_t e = prep(k_yfwd<T, N, VAR>, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.g.kxp / TX, (a.g.nz + NB - 1) / NB, a.nfo);
  k_yfwd<T, N, VAR><<<grid, SH::NTH, smem, s>>>(a);
  return cudaGetLastError();
}
template <typename T, int N>
cudaError_t yfwd_n(const PassArgs& a, cudaStream_t s) {
  PS_SHAPE_DISPATCH(yfwd_nv, a.shape[1], a, s);
}
template <typename T, int N, int VAR = 0>
cudaError_t zfwd_nv(const PassArgs& a0, cudaStream_t s) {
  PassArgs a = a0;
  prepare_args(a);
  using V = typename cplx<T>::type;
  using SH = ColShape<T, N, 2, VAR>;
  constexpr int TX = SH::TX, NB = SH::NB;
  const size_t smem = (size_t)ColBuf<T, N>::v * NB * N * TX * sizeof(V);
  cudaError_t e = prep(k_zfwd<T, N, VAR>, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.g.kxp / TX, (a.g.cy + NB - 1) / NB, a.nfo);
  k_zfwd<T, N, VAR><<<grid, SH::NTH, smem, s>>>(a);
  return cudaGetLastError();
}
template <typename T, int N>
cudaError_t zfwd_n(const PassArgs& a, cudaStream_t s) {
  PS_SHAPE_DISPATCH(zfwd_nv, a.shape[2], a, s);
}
template <typename T>
cudaError_t update_launch(const PassArgs& a0, cudaStream_t s) {
  PassArgs a = a0;
  prepare_args(a);
  const int full = (a.mode == ZF_RHS || a.mode == ZF_RK4_4 || a.mode == ZF_RK2_2) ? 1 : 0;
  const long long n = full ? (long long)a.g.nz * a.g.ny * rowlen(a.g) : (long long)a.g.cz * a.g.cy * ncols(a.g);
  if (n >= (1LL << 32) - 256) return cudaErrorInvalidValue;  // the kernel indexes modes in 32 bits
  const unsigned blocks = (unsigned)((n + 255) / 256);
  const bool slab = a.g.kx0 != 0 || a.g.ncx != 0 || a.g.rowlen != 0;
  if (slab) k_update<T, 1, 0, true><<<blocks, 256, 0, s>>>(a, full);  // slabs: HD only
  else if (a.ng == 2) k_update<T, 2, 0><<<blocks, 256, 0, s>>>(a, full);
  else if (a.nsc) k_update<T, 1, 1><<<blocks, 256, 0, s>>>(a, full);
  else k_update<T, 1, 0><<<blocks, 256, 0, s>>>(a, full);
  return cudaGetLastError();
}

#define PS_DISPATCH_N(n, CALL)                     \
  switch (n) {                                     \
    case 8: return CALL(8);                        \
    case 16: return CALL(16);                      \
    case 32: return CALL(32);                      \
    case 48: return CALL(48);                      \
    case 64: return CALL(64);                      \
    case 96: return CALL(96);                      \
    case 128: return CALL(128);                    \
    case 192: return CALL(192);                    \
    case 256: return CALL(256);                    \
    case 512: return CALL(512);                    \
    case 1024: return CALL(1024);                  \
    default: return cudaErrorInvalidValue;         \
  }

}  // namespace ps
