// Pointwise MLP of the learned LES closure (5 -> 64 -> 64 -> 6, GELU) on the
// BF16 tensor cores with FP32 accumulation (mma.sync m16n8k16), forward,
// backward and the Adam update.  See include/ps.h (ps_mlp_*).
//
// Parameter vector (FP32): W1 [5][64] | b1 [64] | W2 [64][64] | b2 [64] |
// W3 [64][6] | b3 [6]   (row-major, y = x W + b).
//
// One CTA (4 warps) processes chunks of 128 samples; warp w owns samples
// 32w..32w+31 (two 16-row tiles) for the per-sample products, and rows
// 16w..16w+15 of each weight gradient for the batch-reduction products.
// Operands are rounded to BF16 where they enter a tensor-core product; biases,
// pre-activations, GELU and all accumulations stay FP32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>

#include "ps.h"
#include "ps_tb.cuh"

namespace ps {
void set_last_error(const std::string& msg);
}

namespace {

constexpr int H = 64, NI = 5, NO = 6;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NI * H, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + H * NO, NPARAM = OFF_B3 + NO;
static_assert(NPARAM == PS_MLP_NPARAM, "parameter layout");
constexpr int CH = 128;  // samples per chunk
constexpr float C_GELU = 0.7978845608028654f;  // sqrt(2/pi)

typedef __nv_bfloat16 bf;

__device__ __forceinline__ float gelu(float x) {
  return 0.5f * x * (1.f + tanhf(C_GELU * (x + 0.044715f * x * x * x)));
}
__device__ __forceinline__ float gelu_grad(float x) {
  const float t = tanhf(C_GELU * (x + 0.044715f * x * x * x));
  return 0.5f * (1.f + t) + 0.5f * x * (1.f - t * t) * C_GELU * (1.f + 3.f * 0.044715f * x * x);
}

__device__ __forceinline__ uint32_t pack(bf lo, bf hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// D += A (16x16, bf16) * B (16x8, bf16), FP32 accumulate.
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// A fragment of the 16x16 tile at (r0, k0) of a matrix given by an accessor
// at(row, col) (PTX m16n8k16 layout: lane l holds rows l/4 and l/4+8, columns
// 2(l%4)+{0,1} and +8).
template <class F>
__device__ __forceinline__ void load_a(uint32_t (&a)[4], F at, int r0, int k0) {
  const int l = threadIdx.x & 31, r = r0 + l / 4, c = k0 + 2 * (l % 4);
  a[0] = pack(at(r, c), at(r, c + 1));
  a[1] = pack(at(r + 8, c), at(r + 8, c + 1));
  a[2] = pack(at(r, c + 8), at(r, c + 9));
  a[3] = pack(at(r + 8, c + 8), at(r + 8, c + 9));
}
// B fragment of the 16x8 tile at (k0, n0) of a K x N matrix at(k, n): lane l
// holds column n0 + l/4, rows 2(l%4)+{0,1} and +8.
template <class F>
__device__ __forceinline__ void load_b(uint32_t (&b)[2], F at, int k0, int n0) {
  const int l = threadIdx.x & 31, n = n0 + l / 4, k = k0 + 2 * (l % 4);
  b[0] = pack(at(k, n), at(k + 1, n));
  b[1] = pack(at(k + 8, n), at(k + 9, n));
}
// Visits the accumulator elements of a 16x8 tile: f(row, col, value index).
template <class F>
__device__ __forceinline__ void for_acc(int r0, int n0, F f) {
  const int l = threadIdx.x & 31, r = r0 + l / 4, c = n0 + 2 * (l % 4);
  f(r, c, 0);
  f(r, c + 1, 1);
  f(r + 8, c, 2);
  f(r + 8, c + 1, 3);
}

struct Smem {
  bf w1[16][H];   // W1 padded to 16 input rows (rows 5..15 zero)
  bf w2[H][H];
  bf w3[H][8];    // W3 padded to 8 outputs
  float b1[H], b2[H], b3[8];
  bf x[CH][16];   // inputs padded to 16
  bf h1[CH][H], h2[CH][H];
  float z1[CH][H], z2[CH][H];
  bf dy[CH][16];  // output deltas padded to 16 (columns 6..15 zero)
  bf dz1[CH][H], dz2[CH][H];
  float yf[CH][8];  // network outputs (tensor-basis fit)
};

__device__ void load_weights(Smem& s, const float* __restrict__ p) {
  for (int i = threadIdx.x; i < 16 * H; i += blockDim.x) {
    const int r = i / H, c = i % H;
    s.w1[r][c] = __float2bfloat16(r < NI ? p[OFF_W1 + r * H + c] : 0.f);
  }
  for (int i = threadIdx.x; i < H * H; i += blockDim.x) s.w2[i / H][i % H] = __float2bfloat16(p[OFF_W2 + i]);
  for (int i = threadIdx.x; i < H * 8; i += blockDim.x) {
    const int r = i / 8, c = i % 8;
    s.w3[r][c] = __float2bfloat16(c < NO ? p[OFF_W3 + r * NO + c] : 0.f);
  }
  for (int i = threadIdx.x; i < H; i += blockDim.x) {
    s.b1[i] = p[OFF_B1 + i];
    s.b2[i] = p[OFF_B2 + i];
  }
  if (threadIdx.x < 8) s.b3[threadIdx.x] = threadIdx.x < NO ? p[OFF_B3 + threadIdx.x] : 0.f;
}

// Forward pass of the warp's two 16-sample tiles of the chunk; y (FP32,
// count x 6) is written for samples < count when yout != null.
__device__ void forward_tiles(Smem& s, int count, float* yout, float (*yreg)[4]) {
  const int w = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const int r0 = 32 * w + 16 * t;
    uint32_t a[4];
    // layer 1: z1 = x W1 + b1
    load_a(a, [&](int r, int c) { return s.x[r][c]; }, r0, 0);
#pragma unroll
    for (int nt = 0; nt < H / 8; ++nt) {
      float d[4] = {0, 0, 0, 0};
      uint32_t b[2];
      load_b(b, [&](int k, int n) { return s.w1[k][n]; }, 0, 8 * nt);
      mma16816(d, a, b);
      for_acc(r0, 8 * nt, [&](int r, int c, int i) {
        const float z = d[i] + s.b1[c];
        s.z1[r][c] = z;
        s.h1[r][c] = __float2bfloat16(gelu(z));
      });
    }
    __syncwarp();
    // layer 2: z2 = h1 W2 + b2
    float acc[H / 8][4];
#pragma unroll
    for (int nt = 0; nt < H / 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
    for (int kt = 0; kt < H / 16; ++kt) {
      load_a(a, [&](int r, int c) { return s.h1[r][c]; }, r0, 16 * kt);
#pragma unroll
      for (int nt = 0; nt < H / 8; ++nt) {
        uint32_t b[2];
        load_b(b, [&](int k, int n) { return s.w2[k][n]; }, 16 * kt, 8 * nt);
        mma16816(acc[nt], a, b);
      }
    }
#pragma unroll
    for (int nt = 0; nt < H / 8; ++nt)
      for_acc(r0, 8 * nt, [&](int r, int c, int i) {
        const float z = acc[nt][i] + s.b2[c];
        s.z2[r][c] = z;
        s.h2[r][c] = __float2bfloat16(gelu(z));
      });
    __syncwarp();
    // layer 3: y = h2 W3 + b3
    float d[4] = {0, 0, 0, 0};
#pragma unroll
    for (int kt = 0; kt < H / 16; ++kt) {
      load_a(a, [&](int r, int c) { return s.h2[r][c]; }, r0, 16 * kt);
      uint32_t b[2];
      load_b(b, [&](int k, int n) { return s.w3[k][n]; }, 16 * kt, 0);
      mma16816(d, a, b);
    }
    for_acc(r0, 0, [&](int r, int c, int i) {
      const float y = d[i] + s.b3[c];
      yreg[t][i] = y;
      if (yout && c < NO && r < count) yout[r * NO + c] = y;
    });
  }
}

__device__ void stage_inputs(Smem& s, const float* __restrict__ X, int count) {
  for (int i = threadIdx.x; i < CH * 16; i += blockDim.x) {
    const int r = i / 16, c = i % 16;
    s.x[r][c] = __float2bfloat16((r < count && c < NI) ? X[r * NI + c] : 0.f);
  }
}

// Inference: each warp keeps the whole network's BF16 weight fragments and its
// biases in registers and runs 16-sample tiles through it.  The m16n8
// accumulator fragments of two neighbouring 8-column tiles of one layer are,
// after bias, GELU and BF16 packing, exactly the m16n8k16 A fragment of the
// next layer's 16-column k tile, so activations never leave the registers.
// Same products, roundings and summation order as forward_tiles.
__global__ void __launch_bounds__(128) k_mlp_forward(const float* __restrict__ p, const float* __restrict__ X,
                                                     float* __restrict__ Y, long long B) {
  const int lane = threadIdx.x & 31;
  const int qd = lane & 3, rq = lane >> 2;  // column pair and row within a fragment
  // B fragments: W[k][n] at k = k0 + 2 qd + {0, 1} (+ 8), n = n0 + rq
  auto wfrag = [&](int off, int K, int N, int k0, int n0, uint32_t (&b)[2]) {
    const int n = n0 + rq, k = k0 + 2 * qd;
    auto w = [&](int kk) { return __float2bfloat16((kk < K && n < N) ? p[off + kk * N + n] : 0.f); };
    b[0] = pack(w(k), w(k + 1));
    b[1] = pack(w(k + 8), w(k + 9));
  };
  uint32_t w1[H / 8][2], w2[H / 16][H / 8][2], w3[H / 16][2];
#pragma unroll
  for (int nt = 0; nt < H / 8; ++nt) wfrag(OFF_W1, NI, H, 0, 8 * nt, w1[nt]);
#pragma unroll
  for (int kt = 0; kt < H / 16; ++kt) {
#pragma unroll
    for (int nt = 0; nt < H / 8; ++nt) wfrag(OFF_W2, H, H, 16 * kt, 8 * nt, w2[kt][nt]);
    wfrag(OFF_W3, H, NO, 16 * kt, 0, w3[kt]);
  }
  float bb1[H / 8][2], bb2[H / 8][2], bb3[2];
#pragma unroll
  for (int nt = 0; nt < H / 8; ++nt)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      bb1[nt][j] = p[OFF_B1 + 8 * nt + 2 * qd + j];
      bb2[nt][j] = p[OFF_B2 + 8 * nt + 2 * qd + j];
    }
#pragma unroll
  for (int j = 0; j < 2; ++j) bb3[j] = 2 * qd + j < NO ? p[OFF_B3 + 2 * qd + j] : 0.f;
  const long long ntiles = (B + 15) / 16;
  const long long wstride = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long tile = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); tile < ntiles;
       tile += wstride) {
    const long long r0 = tile * 16 + rq, r1 = r0 + 8;
    // layer 1 input fragment: columns 2 qd + {0, 1} of the 5 inputs (k tile 0)
    auto xin = [&](long long r, int c) { return __float2bfloat16((r < B && c < NI) ? X[r * NI + c] : 0.f); };
    uint32_t a[4];
    a[0] = pack(xin(r0, 2 * qd), xin(r0, 2 * qd + 1));
    a[1] = pack(xin(r1, 2 * qd), xin(r1, 2 * qd + 1));
    a[2] = a[3] = 0u;
    // layers 1 and 2
    uint32_t h[H / 16][4];
#pragma unroll
    for (int nt = 0; nt < H / 8; ++nt) {
      float d[4] = {0, 0, 0, 0};
      mma16816(d, a, w1[nt]);
      const bf g0 = __float2bfloat16(gelu(d[0] + bb1[nt][0])), g1 = __float2bfloat16(gelu(d[1] + bb1[nt][1]));
      const bf g2 = __float2bfloat16(gelu(d[2] + bb1[nt][0])), g3 = __float2bfloat16(gelu(d[3] + bb1[nt][1]));
      h[nt >> 1][(nt & 1) * 2 + 0] = pack(g0, g1);  // row r0
      h[nt >> 1][(nt & 1) * 2 + 1] = pack(g2, g3);  // row r1
    }
    float acc[H / 8][4];
#pragma unroll
    for (int nt = 0; nt < H / 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
    for (int kt = 0; kt < H / 16; ++kt) {
      const uint32_t ak[4] = {h[kt][0], h[kt][1], h[kt][2], h[kt][3]};
#pragma unroll
      for (int nt = 0; nt < H / 8; ++nt) mma16816(acc[nt], ak, w2[kt][nt]);
    }
#pragma unroll
    for (int nt = 0; nt < H / 8; ++nt) {
      const bf g0 = __float2bfloat16(gelu(acc[nt][0] + bb2[nt][0])), g1 = __float2bfloat16(gelu(acc[nt][1] + bb2[nt][1]));
      const bf g2 = __float2bfloat16(gelu(acc[nt][2] + bb2[nt][0])), g3 = __float2bfloat16(gelu(acc[nt][3] + bb2[nt][1]));
      h[nt >> 1][(nt & 1) * 2 + 0] = pack(g0, g1);
      h[nt >> 1][(nt & 1) * 2 + 1] = pack(g2, g3);
    }
    // layer 3
    float d[4] = {0, 0, 0, 0};
#pragma unroll
    for (int kt = 0; kt < H / 16; ++kt) {
      const uint32_t ak[4] = {h[kt][0], h[kt][1], h[kt][2], h[kt][3]};
      mma16816(d, ak, w3[kt]);
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int c = 2 * qd + j;
      if (c < NO) {
        if (r0 < B) Y[r0 * NO + c] = d[j] + bb3[j];
        if (r1 < B) Y[r1 * NO + c] = d[2 + j] + bb3[j];
      }
    }
  }
}

// Forward + backward over B samples; parameter gradients accumulate
// (atomically) into grad[NPARAM] and the loss into *loss.
//   MODE_PLAIN: mean-squared error of y against T
//   MODE_TB   : mean-squared error of the model stress sum_n y_n T_n(A/s_A)
//               (T_n the tensor basis of the gradient rows Ag[B][9]) against T/s_tau
//   MODE_DY   : no loss; T holds dL/dy per sample (backpropagation only)
enum { MODE_PLAIN = 0, MODE_TB = 1, MODE_DY = 2 };
template <int MODE>
__global__ void __launch_bounds__(128) k_mlp_grad(const float* __restrict__ p, const float* __restrict__ X,
                                                  const float* __restrict__ Ag, const float* __restrict__ T,
                                                  long long B, float inv_sA, float inv_stau, float* grad,
                                                  double* loss) {
  extern __shared__ __align__(16) unsigned char raw[];
  Smem& s = *reinterpret_cast<Smem*>(raw);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  load_weights(s, p);
  const float scale = 2.f / (float)(B * NO);
  double lsum = 0.0;
  // weight-gradient accumulators of this CTA (flushed once, after all chunks):
  // rows 16w..16w+15 of dW2 and dW3, and (warp 0) dW1; column sums of the deltas
  float a1[H / 8][4], a2[H / 8][4], a3[4];
#pragma unroll
  for (int nt = 0; nt < H / 8; ++nt)
#pragma unroll
    for (int i = 0; i < 4; ++i) a1[nt][i] = a2[nt][i] = 0.f;
  a3[0] = a3[1] = a3[2] = a3[3] = 0.f;
  float bsum = 0.f;  // column sum of (dz1 | dz2 | dy) for column threadIdx.x (+128)
  float bsum2 = 0.f;
  for (long long c0 = (long long)blockIdx.x * CH; c0 < B; c0 += (long long)gridDim.x * CH) {
    const int count = (int)(B - c0 < CH ? B - c0 : CH);
    __syncthreads();
    stage_inputs(s, X + c0 * NI, count);
    __syncthreads();
    float yreg[2][4];
    forward_tiles(s, count, nullptr, yreg);
    if constexpr (MODE == MODE_DY) {
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int r0 = 32 * w + 16 * t;
        for_acc(r0, 0, [&](int r, int c, int i) {
          const float dy = (c < NO && r < count) ? T[(c0 + r) * NO + c] : 0.f;
          s.dy[r][c] = __float2bfloat16(dy);
          s.dy[r][c + 8] = __float2bfloat16(0.f);
        });
      }
    } else if constexpr (MODE == MODE_PLAIN) {
      // output delta dy = 2 (y - t)/(B * 6); loss terms
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int r0 = 32 * w + 16 * t;
        for_acc(r0, 0, [&](int r, int c, int i) {
          float dy = 0.f;
          if (c < NO && r < count) {
            const float e = yreg[t][i] - T[(c0 + r) * NO + c];
            lsum += (double)e * e;
            dy = scale * e;
          }
          s.dy[r][c] = __float2bfloat16(dy);
          s.dy[r][c + 8] = __float2bfloat16(0.f);
        });
      }
    } else {
      // gather each sample's six outputs, then one lane per sample:
      // m = Tb^T y, e = m - t/s_tau, dy = 2/(B*6) Tb e
#pragma unroll
      for (int t = 0; t < 2; ++t)
        for_acc(32 * w + 16 * t, 0, [&](int r, int c, int i) { s.yf[r][c] = yreg[t][i]; });
      __syncwarp();
      const int r = 32 * w + lane;
      float dy[NO] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (r < count) {
        float a[3][3];
        const float* ar = Ag + (c0 + r) * 9;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) a[i][j] = ar[3 * i + j];
        float Tb[6][6];
        ps::tensor_basis(a, inv_sA, Tb);
#pragma unroll
        for (int m = 0; m < NO; ++m) {
          float mv = 0.f;
#pragma unroll
          for (int n = 0; n < NO; ++n) mv += Tb[n][m] * s.yf[r][n];
          const float e = mv - T[(c0 + r) * NO + m] * inv_stau;
          lsum += (double)e * e;
#pragma unroll
          for (int n = 0; n < NO; ++n) dy[n] += scale * Tb[n][m] * e;
        }
      }
#pragma unroll
      for (int n = 0; n < 16; ++n) s.dy[r][n] = __float2bfloat16(n < NO ? dy[n] : 0.f);
    }
    __syncwarp();
    // dh2 = dy W3^T, dz2 = dh2 * gelu'(z2)
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int r0 = 32 * w + 16 * t;
      uint32_t a[4];
      load_a(a, [&](int r, int c) { return s.dy[r][c]; }, r0, 0);
#pragma unroll
      for (int nt = 0; nt < H / 8; ++nt) {
        float d[4] = {0, 0, 0, 0};
        uint32_t b[2];
        // B(k = output, n = hidden) = W3[hidden][output], outputs >= 8 are zero
        load_b(b, [&](int k, int n) { return k < 8 ? s.w3[n][k] : __float2bfloat16(0.f); }, 0, 8 * nt);
        mma16816(d, a, b);
        for_acc(r0, 8 * nt, [&](int r, int c, int i) { s.dz2[r][c] = __float2bfloat16(d[i] * gelu_grad(s.z2[r][c])); });
      }
    }
    __syncwarp();
    // dh1 = dz2 W2^T, dz1 = dh1 * gelu'(z1)
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int r0 = 32 * w + 16 * t;
      float acc[H / 8][4];
#pragma unroll
      for (int nt = 0; nt < H / 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
      for (int kt = 0; kt < H / 16; ++kt) {
        uint32_t a[4];
        load_a(a, [&](int r, int c) { return s.dz2[r][c]; }, r0, 16 * kt);
#pragma unroll
        for (int nt = 0; nt < H / 8; ++nt) {
          uint32_t b[2];
          load_b(b, [&](int k, int n) { return s.w2[n][k]; }, 16 * kt, 8 * nt);  // W2^T
          mma16816(acc[nt], a, b);
        }
      }
#pragma unroll
      for (int nt = 0; nt < H / 8; ++nt)
        for_acc(r0, 8 * nt, [&](int r, int c, int i) { s.dz1[r][c] = __float2bfloat16(acc[nt][i] * gelu_grad(s.z1[r][c])); });
    }
    __syncthreads();
    // weight gradients: rows 16w..16w+15 of dW = A^T D over the chunk's samples
    // dW2[i][j] = sum_s h1[s][i] dz2[s][j];  dW1[i][j] = sum_s x[s][i] dz1[s][j] (w = 0 only)
    // dW3[i][o] = sum_s h2[s][i] dy[s][o]
    {
      const int m0 = 16 * w;
#pragma unroll
      for (int kt = 0; kt < CH / 16; ++kt) {
        uint32_t a[4], b[2];
        load_a(a, [&](int r, int c) { return s.h1[c][r]; }, m0, 16 * kt);
#pragma unroll
        for (int nt = 0; nt < H / 8; ++nt) {
          load_b(b, [&](int k, int n) { return s.dz2[k][n]; }, 16 * kt, 8 * nt);
          mma16816(a2[nt], a, b);
        }
        load_a(a, [&](int r, int c) { return s.h2[c][r]; }, m0, 16 * kt);
        load_b(b, [&](int k, int n) { return s.dy[k][n]; }, 16 * kt, 0);
        mma16816(a3, a, b);
      }
      if (w == 0) {
#pragma unroll
        for (int kt = 0; kt < CH / 16; ++kt) {
          uint32_t a[4], b[2];
          load_a(a, [&](int r, int c) { return s.x[c][r]; }, 0, 16 * kt);
#pragma unroll
          for (int nt = 0; nt < H / 8; ++nt) {
            load_b(b, [&](int k, int n) { return s.dz1[k][n]; }, 16 * kt, 8 * nt);
            mma16816(a1[nt], a, b);
          }
        }
      }
    }
    // bias gradients: column sums of the deltas as stored (BF16), like the
    // weight gradients that use them
    {
      const int c = threadIdx.x;  // 0..127: dz1 (c < 64) or dz2 (c >= 64)
      for (int r = 0; r < count; ++r) bsum += __bfloat162float(c < H ? s.dz1[r][c] : s.dz2[r][c - H]);
      if (c < NO)
        for (int r = 0; r < count; ++r) bsum2 += __bfloat162float(s.dy[r][c]);
    }
  }
  // flush this CTA's gradients
  {
    const int m0 = 16 * w;
#pragma unroll
    for (int nt = 0; nt < H / 8; ++nt)
      for_acc(m0, 8 * nt, [&](int r, int c, int i) { atomicAdd(grad + OFF_W2 + r * H + c, a2[nt][i]); });
    for_acc(m0, 0, [&](int r, int c, int i) {
      if (c < NO) atomicAdd(grad + OFF_W3 + r * NO + c, a3[i]);
    });
    if (w == 0) {
#pragma unroll
      for (int nt = 0; nt < H / 8; ++nt)
        for_acc(0, 8 * nt, [&](int r, int c, int i) {
          if (r < NI) atomicAdd(grad + OFF_W1 + r * H + c, a1[nt][i]);
        });
    }
    const int c = threadIdx.x;
    atomicAdd(grad + (c < H ? OFF_B1 + c : OFF_B2 + c - H), bsum);
    if (c < NO) atomicAdd(grad + OFF_B3 + c, bsum2);
  }
  // loss
  if constexpr (MODE != MODE_DY) {
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0) atomicAdd(loss, lsum / (double)(B * NO));
  }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

int grid_for(long long B) {
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long chunks = (B + CH - 1) / CH;
  const long long g = 2LL * nsm;
  return (int)(chunks < g ? chunks : g);
}

ps_status cuerr(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PS_OK;
  ps::set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
  return PS_ERR_CUDA;
}

}  // namespace

extern "C" {

ps_status ps_mlp_forward(const float* params, const float* X, float* Y, long long count, void* stream) {
  if (!params || !X || !Y || count < 0) {
    ps::set_last_error("ps_mlp_forward: NULL buffer or negative count");
    return PS_ERR_INVALID_ARG;
  }
  if (count == 0) return PS_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_mlp_forward<<<grid_for(count), 128, 0, s>>>(params, X, Y, count);
  return cuerr(cudaGetLastError(), "ps_mlp_forward");
}

ps_status ps_mlp_grad(const float* params, const float* X, const float* T, long long count, float* grad,
                      double* loss, void* stream) {
  if (!params || !X || !T || !grad || !loss || count <= 0) {
    ps::set_last_error("ps_mlp_grad: NULL buffer or non-positive count");
    return PS_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(float) * NPARAM, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(double), s);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_mlp_grad<MODE_PLAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
  if (e != cudaSuccess) return cuerr(e, "ps_mlp_grad");
  k_mlp_grad<MODE_PLAIN><<<grid_for(count), 128, sizeof(Smem), s>>>(params, X, nullptr, T, count, 1.f, 1.f, grad, loss);
  return cuerr(cudaGetLastError(), "ps_mlp_grad");
}

ps_status ps_mlp_grad_tb(const float* params, const float* X, const float* A, const float* T, long long count,
                         double s_A, double s_tau, float* grad, double* loss, void* stream) {
  if (!params || !X || !A || !T || !grad || !loss || count <= 0) {
    ps::set_last_error("ps_mlp_grad_tb: NULL buffer or non-positive count");
    return PS_ERR_INVALID_ARG;
  }
  if (!(s_A > 0) || !(s_tau > 0) || !std::isfinite(s_A) || !std::isfinite(s_tau)) {
    ps::set_last_error("ps_mlp_grad_tb: scales must be positive and finite");
    return PS_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(float) * NPARAM, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(double), s);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_mlp_grad<MODE_TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
  if (e != cudaSuccess) return cuerr(e, "ps_mlp_grad_tb");
  k_mlp_grad<MODE_TB><<<grid_for(count), 128, sizeof(Smem), s>>>(params, X, A, T, count, (float)(1.0 / s_A),
                                                              (float)(1.0 / s_tau), grad, loss);
  return cuerr(cudaGetLastError(), "ps_mlp_grad_tb");
}

ps_status ps_mlp_backward(const float* params, const float* X, const float* dY, long long count, float* grad,
                          void* stream) {
  if (!params || !X || !dY || !grad || count < 0) {
    ps::set_last_error("ps_mlp_backward: NULL buffer or negative count");
    return PS_ERR_INVALID_ARG;
  }
  if (count == 0) return PS_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e =
      cudaFuncSetAttribute(k_mlp_grad<MODE_DY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
  if (e != cudaSuccess) return cuerr(e, "ps_mlp_backward");
  k_mlp_grad<MODE_DY><<<grid_for(count), 128, sizeof(Smem), s>>>(params, X, nullptr, dY, count, 1.f, 1.f, grad,
                                                                 nullptr);
  return cuerr(cudaGetLastError(), "ps_mlp_backward");
}

ps_status ps_mlp_adam(float* params, const float* grad, float* m, float* v, int step, float lr, float beta1,
                      float beta2, float eps, void* stream) {
  if (!params || !grad || !m || !v || step < 1) {
    ps::set_last_error("ps_mlp_adam: NULL buffer or step < 1");
    return PS_ERR_INVALID_ARG;
  }
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  k_adam<<<(NPARAM + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(params, grad, m, v, NPARAM, lr,
                                                                             beta1, beta2, eps, c1, c2);
  return cuerr(cudaGetLastError(), "ps_mlp_adam");
}

}  // extern "C"
