// Per-joint steps of the learned preconditioner's application
// M^{-1} = C^T G^T G C, G = diag(s) (I - A) (k_lpc.cu has the form), shared by
// the one-launch-per-step kernels of k_lpc.cu and the persistent PCG kernel
// of k_pcg32.cu.  Vectors are [5][K] (rows 0-2 used).
#pragma once
#include "mabd_internal.h"

namespace mabd {

// y_k = s_k (t_k - sum_{lower e} alpha_e E_e t_n)
__device__ __forceinline__ void lpc_y_one(const LpcGraph &G, const LpcAct &A, const float *t, float *y, int k) {
  const int K = G.K;
  float v[3] = {t[k], t[(size_t)K + k], t[2 * (size_t)K + k]};
  for (int e = G.off[k]; e < G.off[k + 1]; ++e) {
    const int n = G.nbr[e];
    if (n >= k) continue;
    const float al = A.alpha[e];
    const float *Ee = A.E + (size_t)LPC_ES * e;
    const float tn[3] = {t[n], t[(size_t)K + n], t[2 * (size_t)K + n]};
#pragma unroll
    for (int r = 0; r < 3; ++r) v[r] -= al * (Ee[3 * r] * tn[0] + Ee[3 * r + 1] * tn[1] + Ee[3 * r + 2] * tn[2]);
  }
  const float sk = A.s[k];
#pragma unroll
  for (int r = 0; r < 3; ++r) y[(size_t)r * K + k] = sk * v[r];
}

// z_k = C_k^T (s_k y_k - sum_{upper e} alpha_rev(e) E_e s_n y_n); returns r_k . z_k
__device__ __forceinline__ float lpc_z_one(const LpcGraph &G, const LpcAct &A, const float *y, const float *r,
                                           float *z, int k) {
  const int K = G.K;
  const float sk = A.s[k];
  float u[3] = {sk * y[k], sk * y[(size_t)K + k], sk * y[2 * (size_t)K + k]};
  for (int e = G.off[k]; e < G.off[k + 1]; ++e) {
    const int n = G.nbr[e];
    if (n <= k) continue;
    const float al = A.alpha[G.rev[e]] * A.s[n];
    const float *Ee = A.E + (size_t)LPC_ES * e;
    const float yn[3] = {y[n], y[(size_t)K + n], y[2 * (size_t)K + n]};
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] -= al * (Ee[3 * c] * yn[0] + Ee[3 * c + 1] * yn[1] + Ee[3 * c + 2] * yn[2]);
  }
  const float *Cp = A.C + (size_t)6 * k;
  // z = C^T u with C packed lower (c00 c10 c11 c20 c21 c22)
  const float z0 = Cp[0] * u[0] + Cp[1] * u[1] + Cp[3] * u[2];
  const float z1 = Cp[2] * u[1] + Cp[4] * u[2];
  const float z2 = Cp[5] * u[2];
  z[k] = z0;
  z[(size_t)K + k] = z1;
  z[2 * (size_t)K + k] = z2;
  z[3 * (size_t)K + k] = 0.f;
  z[4 * (size_t)K + k] = 0.f;
  return r[k] * z0 + r[(size_t)K + k] * z1 + r[2 * (size_t)K + k] * z2;
}

}  // namespace mabd
