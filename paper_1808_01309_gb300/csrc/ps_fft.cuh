// Line-FFT building blocks for the pseudospectral passes (sm_103a).
//
// One length-N line is spread over G = N/E threads; the thread with index j0
// holds the E elements n = j0 + m*(N/E), m = 0..E-1, in registers.  A
// mixed-radix Stockham autosort FFT (Stockham 1966; Cooley-Tukey stages with a
// self-sorting output order) runs one stage per radix R: the thread does E/R
// radix-R butterflies on its registers, multiplies by the stage twiddles and,
// between stages, exchanges elements through shared memory.  The first stage
// reads, and the last stage leaves, exactly the elements n = j0 + m*(N/E), so
// the passes load straight from HBM into registers and store straight back:
// the strided z/y passes are coalesced across neighbouring lines (kx columns),
// the x pass along the row.
//
// Transform convention (Sec. 2, Eq. fftsum): forward X[k] = sum_n x[n]
// exp(-2 pi i k n/N) (DIR = -1), backward with exp(+2 pi i k n/N) (DIR = +1),
// both unnormalised; the 1/(Nx Ny Nz) of the forward transform is applied once
// in the last forward pass.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ps {

template <typename T> struct cplx;
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<double> { using type = double2; };

template <typename V> __device__ __forceinline__ V mk(decltype(V::x) x, decltype(V::x) y) { V v; v.x = x; v.y = y; return v; }
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return mk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return mk<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return mk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) {
  return mk<V>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename V> __device__ __forceinline__ V cconj(V a) { return mk<V>(a.x, -a.y); }
template <typename V> __device__ __forceinline__ V cscale(V a, decltype(V::x) s) { return mk<V>(a.x * s, a.y * s); }
template <typename V> __device__ __forceinline__ V czero() { return mk<V>(0, 0); }
// i * a and -i * a
template <typename V> __device__ __forceinline__ V cmul_i(V a) { return mk<V>(-a.y, a.x); }
template <typename V> __device__ __forceinline__ V cmul_mi(V a) { return mk<V>(a.y, -a.x); }

// FP32 complex add, subtract and real scaling as packed two-lane FP32
// instructions (add/sub/mul.rn.f32x2 of sm_100 and later): one instruction per
// complex operation instead of two.
#ifndef PS_F32X2
#define PS_F32X2 1
#endif
#if PS_F32X2
union F2U {
  float2 f;
  unsigned long long u;
};
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  F2U x{a}, y{b}, r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.u) : "l"(x.u), "l"(y.u));
  return r.f;
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  F2U x{a}, y{b}, r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.u) : "l"(x.u), "l"(y.u));
  return r.f;
}
__device__ __forceinline__ float2 cscale(float2 a, float s) {
  F2U x{a}, y{make_float2(s, s)}, r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.u) : "l"(x.u), "l"(y.u));
  return r.f;
}
#endif

// Multiply by exp(DIR * 2 pi i * s/16) for a compile-time s in [0, 8).
// cos(pi/8), sin(pi/8) and sqrt(1/2) are the exact mathematical constants,
// rounded by the compiler to the working precision.
template <int S16, int DIR, typename V>
__device__ __forceinline__ V rot16(V v) {
  using T = decltype(V::x);
  constexpr double C1 = 0.92387953251128675612818318939678828682;  // cos(pi/8)
  constexpr double S1 = 0.38268343236508977172845998403039886676;  // sin(pi/8)
  constexpr double H = 0.70710678118654752440084436210484903928;   // sqrt(1/2)
  if constexpr (S16 == 0) {
    return v;
  } else if constexpr (S16 == 4) {
    return DIR > 0 ? cmul_i(v) : cmul_mi(v);
  } else if constexpr (S16 == 2) {  // (1 + DIR i)/sqrt2
    return DIR > 0 ? mk<V>(T(H) * (v.x - v.y), T(H) * (v.x + v.y))
                   : mk<V>(T(H) * (v.x + v.y), T(H) * (v.y - v.x));
  } else if constexpr (S16 == 6) {  // (-1 + DIR i)/sqrt2
    return DIR > 0 ? mk<V>(-T(H) * (v.x + v.y), T(H) * (v.x - v.y))
                   : mk<V>(T(H) * (v.y - v.x), -T(H) * (v.x + v.y));
  } else {
    constexpr double c = (S16 == 1) ? C1 : (S16 == 3) ? S1 : (S16 == 5) ? -S1 : -C1;
    constexpr double s = (S16 == 1) ? S1 : (S16 == 3) ? C1 : (S16 == 5) ? C1 : S1;
    return cmul(v, mk<V>(T(c), T(DIR * s)));
  }
}

template <int B> struct ilog2 { static constexpr int v = 1 + ilog2<B / 2>::v; };
template <> struct ilog2<1> { static constexpr int v = 0; };

__host__ __device__ constexpr int bitrev(int x, int bits) {
  int r = 0;
  for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1) << (bits - 1 - i);
  return r;
}

// In-register DFT of a power-of-two size R in {2,4,8,16}: radix-2 decimation
// in time over a bit-reversed copy; all indices are compile-time after
// unrolling.
template <int R, int DIR, typename V>
__device__ __forceinline__ void dft_pow2(V (&x)[R]) {
  constexpr int L = ilog2<R>::v;
  V y[R];
#pragma unroll
  for (int i = 0; i < R; ++i) y[i] = x[bitrev(i, L)];
#pragma unroll
  for (int len = 2; len <= R; len *= 2) {
#pragma unroll
    for (int i = 0; i < R; i += len) {
#pragma unroll
      for (int j = 0; j < len / 2; ++j) {
        V u = y[i + j];
        V v = y[i + j + len / 2];
        // twiddle exp(DIR 2 pi i j/len) = exp(DIR 2 pi i (16 j/len)/16)
        switch ((16 / len) * j) {
          case 0: break;
          case 1: v = rot16<1, DIR>(v); break;
          case 2: v = rot16<2, DIR>(v); break;
          case 3: v = rot16<3, DIR>(v); break;
          case 4: v = rot16<4, DIR>(v); break;
          case 5: v = rot16<5, DIR>(v); break;
          case 6: v = rot16<6, DIR>(v); break;
          case 7: v = rot16<7, DIR>(v); break;
        }
        y[i + j] = cadd(u, v);
        y[i + j + len / 2] = csub(u, v);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < R; ++i) x[i] = y[i];
}

// 3-point DFT: with s = DIR sqrt(3)/2,
//   y0 = x0 + x1 + x2,  y1,2 = x0 - (x1 + x2)/2 +- i s (x1 - x2).
template <int DIR, typename V>
__device__ __forceinline__ void dft3(V& a, V& b, V& c) {
  using T = decltype(V::x);
  constexpr double S3 = 0.86602540378443864676372317075293618347;  // sqrt(3)/2
  const V t1 = cadd(b, c);
  const V t2 = csub(a, cscale(t1, T(0.5)));
  const V d = cscale(csub(b, c), T(DIR * S3));
  a = cadd(a, t1);
  b = cadd(t2, cmul_i(d));
  c = csub(t2, cmul_i(d));
}

// In-register DFT of size R in {2,3,4,6,8,16}.  R = 6 = 2 x 3: two 3-point
// DFTs of the even and odd samples, then X[k] = A0[k] + w6^k A1[k] and
// X[k+3] = A0[k] - w6^k A1[k], w6 = exp(DIR i pi/3).
template <int R, int DIR, typename V>
__device__ __forceinline__ void dft(V (&x)[R]) {
  if constexpr (R == 3) {
    dft3<DIR>(x[0], x[1], x[2]);
  } else if constexpr (R == 6) {
    using T = decltype(V::x);
    constexpr double S3 = 0.86602540378443864676372317075293618347;
    V e0 = x[0], e1 = x[2], e2 = x[4], o0 = x[1], o1 = x[3], o2 = x[5];
    dft3<DIR>(e0, e1, e2);
    dft3<DIR>(o0, o1, o2);
    o1 = cmul(o1, mk<V>(T(0.5), T(DIR * S3)));   // w6
    o2 = cmul(o2, mk<V>(T(-0.5), T(DIR * S3)));  // w6^2
    x[0] = cadd(e0, o0);
    x[3] = csub(e0, o0);
    x[1] = cadd(e1, o1);
    x[4] = csub(e1, o1);
    x[2] = cadd(e2, o2);
    x[5] = csub(e2, o2);
  } else {
    dft_pow2<R, DIR>(x);
  }
}

// Radix schedule per length N and registers per thread E: stage radices
// R0..R3 (1 = no stage).  E = 16 shortens the wider FP32 transforms by one
// shared-memory exchange; E = 8 keeps FP64 within the register file.
template <int N, int E> struct Sched;
template <> struct Sched<8, 8> { static constexpr int S = 1, R0 = 8, R1 = 1, R2 = 1, R3 = 1; };
template <> struct Sched<16, 16> { static constexpr int S = 1, R0 = 16, R1 = 1, R2 = 1, R3 = 1; };
template <> struct Sched<16, 8> { static constexpr int S = 2, R0 = 8, R1 = 2, R2 = 1, R3 = 1; };
template <> struct Sched<32, 8> { static constexpr int S = 2, R0 = 8, R1 = 4, R2 = 1, R3 = 1; };
template <> struct Sched<64, 8> { static constexpr int S = 2, R0 = 8, R1 = 8, R2 = 1, R3 = 1; };
template <> struct Sched<64, 16> { static constexpr int S = 2, R0 = 16, R1 = 4, R2 = 1, R3 = 1; };
template <> struct Sched<128, 16> { static constexpr int S = 2, R0 = 16, R1 = 8, R2 = 1, R3 = 1; };
template <> struct Sched<128, 8> { static constexpr int S = 3, R0 = 8, R1 = 8, R2 = 2, R3 = 1; };
template <> struct Sched<256, 16> { static constexpr int S = 2, R0 = 16, R1 = 16, R2 = 1, R3 = 1; };
template <> struct Sched<256, 8> { static constexpr int S = 3, R0 = 8, R1 = 8, R2 = 4, R3 = 1; };
template <> struct Sched<512, 8> { static constexpr int S = 3, R0 = 8, R1 = 8, R2 = 8, R3 = 1; };
template <> struct Sched<1024, 16> { static constexpr int S = 3, R0 = 16, R1 = 8, R2 = 8, R3 = 1; };
template <> struct Sched<1024, 8> { static constexpr int S = 4, R0 = 8, R1 = 8, R2 = 8, R3 = 2; };
// lengths with a factor 3 (E = 12)
template <> struct Sched<48, 12> { static constexpr int S = 3, R0 = 6, R1 = 4, R2 = 2, R3 = 1; };
template <> struct Sched<96, 12> { static constexpr int S = 3, R0 = 6, R1 = 4, R2 = 4, R3 = 1; };
template <> struct Sched<192, 12> { static constexpr int S = 4, R0 = 6, R1 = 4, R2 = 4, R3 = 2; };

// Registers per thread for a length-N line in precision T.
template <typename T, int N> struct EOf {
  static constexpr int v = (N % 3 == 0) ? 12
                           : (sizeof(T) == 4 && (N == 16 || N == 128 || N == 256 || N == 1024)) ? 16 : 8;
};

// Twiddle tables tw[m] = exp(-2 pi i m/N): read-only global memory (through
// the non-coherent path) or a copy in shared memory.  at<NS, R>(r, b, idx)
// returns the twiddle of input r of the thread's butterfly b in the stage with
// previous radix product NS, which is tw[idx].
template <typename V>
struct GlobalTw {
  const V* __restrict__ p;
  __device__ __forceinline__ V operator[](int i) const { return __ldg(p + i); }
  template <int NS, int R>
  __device__ __forceinline__ V at(int, int, int idx) const { return __ldg(p + idx); }
};
template <typename V>
struct SharedTw {
  const V* p;
  __device__ __forceinline__ V operator[](int i) const { return p[i]; }
  template <int NS, int R>
  __device__ __forceinline__ V at(int, int, int idx) const { return p[idx]; }
};

// Per-thread twiddle slots: stage s > 0 of a schedule needs (E/R_s)(R_s - 1)
// twiddles per thread (inputs r = 1..R_s-1 of each of its butterflies).
template <int N, int E> struct TwSlots {
  using S = Sched<N, E>;
  static constexpr int n1 = S::S > 1 ? (E / S::R1) * (S::R1 - 1) : 0;
  static constexpr int n2 = S::S > 2 ? (E / S::R2) * (S::R2 - 1) : 0;
  static constexpr int n3 = S::S > 3 ? (E / S::R3) * (S::R3 - 1) : 0;
  static constexpr int total = n1 + n2 + n3;
  __host__ __device__ static constexpr int base(int ns) {
    return ns == S::R0 ? 0 : ns == S::R0 * S::R1 ? n1 : n1 + n2;
  }
};

// Twiddles of one thread position j0 gathered into a table [slot][N/E] (slot
// = stage base + b (R-1) + r - 1), so that the G threads of a line read G
// consecutive entries per twiddle: conflict-free shared-memory reads instead of
// scattered table lookups.  Used by kernels whose threads keep one j0 for many
// lines (the persistent x pass).
template <typename V, int N, int E>
struct ThreadTw {
  const V* p;
  int j0;
  template <int NS, int R>
  __device__ __forceinline__ V at(int r, int b, int) const {
    return p[(TwSlots<N, E>::base(NS) + b * (R - 1) + (r - 1)) * (N / E) + j0];
  }
};

// The same twiddles held in registers for the whole kernel (kernels that keep
// one j0 and whose schedule needs few twiddles per thread).
template <typename V, int N, int E>
struct RegTw {
  V w[TwSlots<N, E>::total > 0 ? TwSlots<N, E>::total : 1];
  template <int NS, int R>
  __device__ __forceinline__ V at(int r, int b, int) const {
    return w[TwSlots<N, E>::base(NS) + b * (R - 1) + (r - 1)];
  }
  template <int NS, int R>
  __device__ __forceinline__ void load_stage(const V* __restrict__ tw, int j0) {
    constexpr int NB = E / R;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int k = (j0 + b * (N / E)) % NS;
#pragma unroll
      for (int r = 1; r < R; ++r) w[TwSlots<N, E>::base(NS) + b * (R - 1) + (r - 1)] = __ldg(tw + r * k * (N / (NS * R)));
    }
  }
  __device__ __forceinline__ void load(const V* __restrict__ tw, int j0) {
    using S = Sched<N, E>;
    if constexpr (S::S > 1) load_stage<S::R0, S::R1>(tw, j0);
    if constexpr (S::S > 2) load_stage<S::R0 * S::R1, S::R2>(tw, j0);
    if constexpr (S::S > 3) load_stage<S::R0 * S::R1 * S::R2, S::R3>(tw, j0);
  }
};

template <int N, int E, int NS, int R, typename V>
__device__ __forceinline__ void fill_stage_tw(V* tab, const V* __restrict__ tw, int j0) {
  constexpr int NB = E / R;
  for (int b = 0; b < NB; ++b) {
    const int k = (j0 + b * (N / E)) % NS;
    for (int r = 1; r < R; ++r)
      tab[(TwSlots<N, E>::base(NS) + b * (R - 1) + (r - 1)) * (N / E) + j0] = tw[r * k * (N / (NS * R))];
  }
}

// Thread j0 (0 <= j0 < N/E) writes its column of the per-thread table.
template <int N, int E, typename V>
__device__ void fill_thread_tw(V* tab, const V* __restrict__ tw, int j0) {
  using S = Sched<N, E>;
  if constexpr (S::S > 1) fill_stage_tw<N, E, S::R0, S::R1>(tab, tw, j0);
  if constexpr (S::S > 2) fill_stage_tw<N, E, S::R0 * S::R1, S::R2>(tab, tw, j0);
  if constexpr (S::S > 3) fill_stage_tw<N, E, S::R0 * S::R1 * S::R2, S::R3>(tab, tw, j0);
}

// Twiddle exp(DIR 2 pi i m/N).
template <int DIR, typename V, class TW>
__device__ __forceinline__ V twiddle(const TW& tw, int idx) {
  V w = tw[idx];
  return DIR > 0 ? cconj(w) : w;
}

// One Stockham stage of radix R on a line of length N whose previous stages
// had total radix NS.  Butterfly j takes x[j + r N/R], multiplies by
// W_{NS R}^{r k} (k = j mod NS), transforms, and writes y[(j-k) R + k + r NS].
// Thread j0 owns butterflies j = j0 + b N/E, b < E/R, whose inputs are its
// registers b + r E/R.  The last stage leaves y[j + r N/R] in the same slots.
template <int N, int E, int R, int NS, int DIR, bool LAST, typename V, class TW, class X>
__device__ __forceinline__ void stage(V (&a)[E], int j0, const TW& tw, X& ex) {
  constexpr int NB = E / R;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = j0 + b * (N / E);
    const int k = j % NS;
    V x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = a[b + r * NB];
    if constexpr (NS > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const V w = tw.template at<NS, R>(r, b, r * k * (N / (NS * R)));
        x[r] = cmul(x[r], DIR > 0 ? cconj(w) : w);
      }
    }
    dft<R, DIR>(x);
    if constexpr (LAST) {
#pragma unroll
      for (int r = 0; r < R; ++r) a[b + r * NB] = x[r];
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) ex.template put<NS, R>((j - k) * R + k + r * NS, x[r]);
    }
  }
  if constexpr (!LAST) {
    ex.sync();
#pragma unroll
    for (int m = 0; m < E; ++m) a[m] = ex.template get<NS, R>(j0 + m * (N / E));
    ex.flip();
  }
}

// Full length-N line transform on the E registers of thread j0 (see header).
// Full length-N line transform with a twiddle accessor (GlobalTw, SharedTw).
template <int N, int E, int DIR, typename V, class TW, class X>
__device__ __forceinline__ void line_fft_tw(V (&a)[E], int j0, const TW& tw, X& ex) {
  using S = Sched<N, E>;
  if constexpr (S::S == 1) {
    stage<N, E, S::R0, 1, DIR, true>(a, j0, tw, ex);
  } else if constexpr (S::S == 2) {
    stage<N, E, S::R0, 1, DIR, false>(a, j0, tw, ex);
    stage<N, E, S::R1, S::R0, DIR, true>(a, j0, tw, ex);
  } else if constexpr (S::S == 3) {
    stage<N, E, S::R0, 1, DIR, false>(a, j0, tw, ex);
    stage<N, E, S::R1, S::R0, DIR, false>(a, j0, tw, ex);
    stage<N, E, S::R2, S::R0 * S::R1, DIR, true>(a, j0, tw, ex);
  } else {
    stage<N, E, S::R0, 1, DIR, false>(a, j0, tw, ex);
    stage<N, E, S::R1, S::R0, DIR, false>(a, j0, tw, ex);
    stage<N, E, S::R2, S::R0 * S::R1, DIR, false>(a, j0, tw, ex);
    stage<N, E, S::R3, S::R0 * S::R1 * S::R2, DIR, true>(a, j0, tw, ex);
  }
}

// Full length-N line transform with twiddles read from global memory.
template <int N, int E, int DIR, typename V, class X>
__device__ __forceinline__ void line_fft(V (&a)[E], int j0, const V* __restrict__ twp, X& ex) {
  const GlobalTw<V> tw{twp};
  line_fft_tw<N, E, DIR>(a, j0, tw, ex);
}

// Shared-memory exchange for lines laid out as columns: element n of line l
// at buf[row(n) * LP + l].  With NBUF = 2 two buffers are used alternately so
// that one barrier per exchange suffices (a buffer is rewritten only after the
// barrier of the following exchange, which every thread passes after finishing
// its reads); with NBUF = 1 a second barrier after the reads frees the single
// buffer.  row(n) flips the lowest bit when bit SW of n is set: the first
// exchange writes rows R1 apart, and this keeps them on alternate bank halves.
template <typename V, int SW, int NBUF = 2>
struct ColumnExchange {
  V* buf;
  int bufsz;
  int lp;
  int l;
  int par;
  __device__ __forceinline__ int row(int n) const { return n ^ ((n >> SW) & 1); }
  template <int NS = 0, int R = 0>
  __device__ __forceinline__ void put(int n, V v) { buf[par * bufsz + row(n) * lp + l] = v; }
  template <int NS = 0, int R = 0>
  __device__ __forceinline__ V get(int n) const { return buf[par * bufsz + row(n) * lp + l]; }
  __device__ __forceinline__ void sync() { __syncthreads(); }
  __device__ __forceinline__ void flip() {
    if constexpr (NBUF == 2) par ^= 1;
    else __syncthreads();
  }
};

// Shared-memory exchange for a line stored as a row of N 8- or 16-byte
// elements.  Element n of the exchange written by a stage with previous radix
// product NS and radix R sits at pos<NS, R>(n) = n XOR swz(n): the swizzle only
// permutes the lowest four bits (one 16-slot window), so the contiguous reads
// of the next stage stay conflict-free, while the strided writes
// (j - k) R + k + r NS of consecutive butterflies j spread over all 16 bank
// pairs:
//   NS = 1       : writes R apart  -> mix bits 4..7 into bits 0..3
//   1 < NS < 16  : writes in runs of NS, runs NS R apart -> mix the run index
//                  into the bits above log2(NS)
//   NS >= 16 or 0: runs of >= 16 consecutive slots, identity (0 = natural order)
template <typename V, int PS_UNUSED = 0>
struct RowExchange {
  V* buf;
  int bufsz;
  int par;
  int bar_id = 0;   // > 0: named barrier of this row's nthr threads
  int nthr = 0;
  template <int NS, int R>
  __device__ __forceinline__ static int pos(int n) {
    if constexpr (NS == 1) {
      return n ^ ((n >> 4) & 15);
    } else if constexpr (NS > 1 && NS < 16) {
      constexpr int LNS = ilog2<NS>::v, LRUN = ilog2<NS * R>::v;
      return n ^ (((n >> LRUN) & (16 / NS - 1)) << LNS);
    } else {
      return n;
    }
  }
  template <int NS = 0, int R = 0>
  __device__ __forceinline__ void put(int n, V v) { buf[par * bufsz + pos<NS, R>(n)] = v; }
  template <int NS = 0, int R = 0>
  __device__ __forceinline__ V get(int n) const { return buf[par * bufsz + pos<NS, R>(n)]; }
  __device__ __forceinline__ void sync() {
    if (bar_id > 0) asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(nthr) : "memory");
    else if (bar_id < 0) __syncwarp();
    else __syncthreads();
  }
  __device__ __forceinline__ void flip() { par ^= 1; }
};

// Exchange for NL lines of one row transformed together (line_fft_rows): line
// l of the row's region at buf + l * lstride, slots permuted as in RowExchange.
// With NBUF = 1 one buffer serves every exchange (a second barrier after the
// reads frees it); NBUF = 2 alternates two buffers bufsz apart.
template <typename V, int NBUF = 1>
struct LinesExchange {
  V* buf;
  int lstride;
  int bufsz;
  int par;
  int bar_id = 0;   // > 0: named barrier of this row's nthr threads; < 0: the row is within a warp
  int nthr = 0;
  template <int NS, int R>
  __device__ __forceinline__ void put(int l, int n, V v) {
    buf[par * bufsz + l * lstride + RowExchange<V>::template pos<NS, R>(n)] = v;
  }
  template <int NS, int R>
  __device__ __forceinline__ V get(int l, int n) const {
    return buf[par * bufsz + l * lstride + RowExchange<V>::template pos<NS, R>(n)];
  }
  __device__ __forceinline__ void sync() {
    if (bar_id > 0) asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(nthr) : "memory");
    else if (bar_id < 0) __syncwarp();
    else __syncthreads();
  }
  __device__ __forceinline__ void flip() {
    if constexpr (NBUF == 2) par ^= 1;
    else sync();
  }
};

// One Stockham stage (as in stage()) applied to NL independent lines held by
// the same threads: the butterflies of all lines are issued together (the
// stage twiddles are shared), then one exchange moves all lines.
template <int N, int E, int R, int NS, int DIR, bool LAST, int NL, typename V, class TW, class X>
__device__ __forceinline__ void stage_rows(V (&a)[NL][E], int j0, const TW& tw, X& ex) {
  constexpr int NB = E / R;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = j0 + b * (N / E);
    const int k = j % NS;
    V w[R];
    if constexpr (NS > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const V t = tw.template at<NS, R>(r, b, r * k * (N / (NS * R)));
        w[r] = DIR > 0 ? cconj(t) : t;
      }
    }
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      V x[R];
#pragma unroll
      for (int r = 0; r < R; ++r) x[r] = a[l][b + r * NB];
      if constexpr (NS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) x[r] = cmul(x[r], w[r]);
      }
      dft<R, DIR>(x);
      if constexpr (LAST) {
#pragma unroll
        for (int r = 0; r < R; ++r) a[l][b + r * NB] = x[r];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) ex.template put<NS, R>(l, (j - k) * R + k + r * NS, x[r]);
      }
    }
  }
  if constexpr (!LAST) {
    ex.sync();
#pragma unroll
    for (int l = 0; l < NL; ++l)
#pragma unroll
      for (int m = 0; m < E; ++m) a[l][m] = ex.template get<NS, R>(l, j0 + m * (N / E));
    ex.flip();
  }
}

// NL line transforms of length N at once (see line_fft_tw).
template <int N, int E, int DIR, int NL, typename V, class TW, class X>
__device__ __forceinline__ void line_fft_rows(V (&a)[NL][E], int j0, const TW& tw, X& ex) {
  using S = Sched<N, E>;
  if constexpr (S::S == 1) {
    stage_rows<N, E, S::R0, 1, DIR, true>(a, j0, tw, ex);
  } else if constexpr (S::S == 2) {
    stage_rows<N, E, S::R0, 1, DIR, false>(a, j0, tw, ex);
    stage_rows<N, E, S::R1, S::R0, DIR, true>(a, j0, tw, ex);
  } else if constexpr (S::S == 3) {
    stage_rows<N, E, S::R0, 1, DIR, false>(a, j0, tw, ex);
    stage_rows<N, E, S::R1, S::R0, DIR, false>(a, j0, tw, ex);
    stage_rows<N, E, S::R2, S::R0 * S::R1, DIR, true>(a, j0, tw, ex);
  } else {
    stage_rows<N, E, S::R0, 1, DIR, false>(a, j0, tw, ex);
    stage_rows<N, E, S::R1, S::R0, DIR, false>(a, j0, tw, ex);
    stage_rows<N, E, S::R2, S::R0 * S::R1, DIR, false>(a, j0, tw, ex);
    stage_rows<N, E, S::R3, S::R0 * S::R1 * S::R2, DIR, true>(a, j0, tw, ex);
  }
}

}  // namespace ps
