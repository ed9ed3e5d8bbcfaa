// Tensor basis of the LES closure: the first six tensors of Pope's (1975)
// integrity basis for a traceless velocity gradient, built from S' = S/s_A and
// R' = R/s_A (S, R the symmetric and antisymmetric parts of A_ij = du_i/dx_j):
//   T1 = S'                   T2 = S'R' - R'S'
//   T3 = S'^2 - tr(S'^2) I/3  T4 = R'^2 - tr(R'^2) I/3
//   T5 = R'S'^2 - S'^2R'      T6 = R'^2S' + S'R'^2 - 2 tr(S'R'^2) I/3
// The model stress is tau = s_tau sum_n g_n T_n with g the network outputs.
// Components are stored in the order 11, 22, 33, 12, 13, 23.
#pragma once

namespace ps {

// Symmetric 3x3 matrix -> 6 components.
__device__ __forceinline__ void sym6(const float (&M)[3][3], float (&o)[6]) {
  o[0] = M[0][0];
  o[1] = M[1][1];
  o[2] = M[2][2];
  o[3] = M[0][1];
  o[4] = M[0][2];
  o[5] = M[1][2];
}

__device__ __forceinline__ void matmul3(const float (&X)[3][3], const float (&Y)[3][3], float (&Z)[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Z[i][j] = X[i][0] * Y[0][j] + X[i][1] * Y[1][j] + X[i][2] * Y[2][j];
}

// a: gradient A[i][j]; T[n][m]: component m of basis tensor n + 1.
__device__ __forceinline__ void tensor_basis(const float (&a)[3][3], float inv_sA, float (&T)[6][6]) {
  float S[3][3], R[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      S[i][j] = 0.5f * inv_sA * (a[i][j] + a[j][i]);
      R[i][j] = 0.5f * inv_sA * (a[i][j] - a[j][i]);
    }
  float S2[3][3], R2[3][3], SR[3][3], RS[3][3], RS2[3][3], S2R[3][3], R2S[3][3], SR2[3][3];
  matmul3(S, S, S2);
  matmul3(R, R, R2);
  matmul3(S, R, SR);
  matmul3(R, S, RS);
  matmul3(R, S2, RS2);
  matmul3(S2, R, S2R);
  matmul3(R2, S, R2S);
  matmul3(S, R2, SR2);
  const float trS2 = S2[0][0] + S2[1][1] + S2[2][2];
  const float trR2 = R2[0][0] + R2[1][1] + R2[2][2];
  const float trSR2 = SR2[0][0] + SR2[1][1] + SR2[2][2];
  float M[3][3];
  sym6(S, T[0]);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) M[i][j] = SR[i][j] - RS[i][j];
  sym6(M, T[1]);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) M[i][j] = S2[i][j] - (i == j ? trS2 * (1.f / 3.f) : 0.f);
  sym6(M, T[2]);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) M[i][j] = R2[i][j] - (i == j ? trR2 * (1.f / 3.f) : 0.f);
  sym6(M, T[3]);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) M[i][j] = RS2[i][j] - S2R[i][j];
  sym6(M, T[4]);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) M[i][j] = R2S[i][j] + SR2[i][j] - (i == j ? trSR2 * (2.f / 3.f) : 0.f);
  sym6(M, T[5]);
}

}  // namespace ps
