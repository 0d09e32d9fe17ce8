// FP32 device helpers of the mixed-precision form: the structured
// Hbar^{-1} and the rest-frame constraint rows of a joint, read from the FP32
// copies of R, the joint points and the hinge frame.
#pragma once
#include "mabd_device.cuh"

namespace mabd {

__device__ __forceinline__ void hinvf_apply(const float h[16], const float v[12], float y[12]) {
  y[0] = h[1] * v[0] + h[2] * v[4] + h[3] * v[8];
  y[4] = h[2] * v[0] + h[4] * v[4] + h[5] * v[8];
  y[8] = h[3] * v[0] + h[5] * v[4] + h[6] * v[8];
  y[1] = h[7] * v[1] + h[8] * v[3];
  y[3] = h[8] * v[1] + h[9] * v[3];
  y[2] = h[10] * v[2] + h[11] * v[6];
  y[6] = h[11] * v[2] + h[12] * v[6];
  y[5] = h[13] * v[5] + h[14] * v[7];
  y[7] = h[14] * v[5] + h[15] * v[7];
  y[9] = h[0] * v[9];
  y[10] = h[0] * v[10];
  y[11] = h[0] * v[11];
}

__device__ __forceinline__ void load_hf(const DevBodies &B, int j, float h[16]) {
#pragma unroll
  for (int i = 0; i < 16; ++i) h[i] = __ldg(B.hinvf + (size_t)i * B.M + j);
}

__device__ __forceinline__ void load_Rf(const DevBodies &B, int j, float R[9]) {
#pragma unroll
  for (int i = 0; i < 9; ++i) R[i] = B.Rf[(size_t)i * B.M + j];
}

__device__ __forceinline__ void load3f(const float *p, int N, int k, float out[3]) {
  out[0] = __ldg(p + k);
  out[1] = __ldg(p + (size_t)N + k);
  out[2] = __ldg(p + 2 * (size_t)N + k);
}

// rows of joint k on its side `side` (body with FP32 rotation R): row r is
// s [p; 1] (x) (R^T d_r) (frozen frame, Eq. pcpq), s = +1 on a, -1 on b.
// Writes directions E, points P and the point index pt[r]; returns C_k.
__device__ __forceinline__ int rows_rest_f(const DevJoints &J, int k, int side, const float R[9],
                                           float E[5][3], float P[2][3], int pt[5]) {
  const int K = J.K;
  const int type = J.type[k];
  const float sgn = side == 0 ? 1.f : -1.f;
  load3f(side == 0 ? J.pa1f : J.pb1f, K, k, P[0]);
  if (type == 0) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
      for (int a = 0; a < 3; ++a) E[r][a] = sgn * R[3 * r + a];
      pt[r] = 0;
    }
    return 3;
  }
  load3f(side == 0 ? J.pa2f : J.pb2f, K, k, P[1]);
  float RH[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) RH[i] = J.RHf[(size_t)i * K + k];
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const int rr = r < 3 ? r : (r == 3 ? 0 : 2);
#pragma unroll
    for (int a = 0; a < 3; ++a)
      E[r][a] = sgn * (R[a] * RH[3 * rr] + R[3 + a] * RH[3 * rr + 1] + R[6 + a] * RH[3 * rr + 2]);
    pt[r] = r < 3 ? 0 : 1;
  }
  return 5;
}

}  // namespace mabd
