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

// rows of joint k on its side `side` (body with FP32 rotation R), from the
// FP32 copies of the joint points and frame: joint_rows_pt<float>; PR[r] and
// WR[r] are row r's point and its translation weight (0 for the universal
// joint's point difference)
template <bool XJ>
__device__ __forceinline__ int rows_pt_f(const DevJoints &J, int k, int side, const float R[9],
                                         float E[5][3], float PR[5][3], float WR[5]) {
  return joint_rows_pt<float, XJ>(J, k, side, R, E, PR, WR);
}

}  // namespace mabd
