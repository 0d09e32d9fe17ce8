// Device helpers of the mixed-precision forms: the structured Hbar^{-1} and
// Hbar products (Eq. abd_final), displacements of rest-frame points, and the
// polar rotation and rest-frame right-hand side in double-float arithmetic
// (ff.h).
#pragma once
#include "mabd_f32.cuh"
#include "ff.h"

namespace mabd {

// y = Hbar^{-1} v with the structured inverse (see mabd_internal.h)
template <typename T>
__device__ __forceinline__ void hinv_apply_t(const T h[16], const T v[12], T y[12]) {
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

__device__ __forceinline__ void load_hinvf(const DevBodies &B, int j, float h[16]) {
#pragma unroll
  for (int i = 0; i < 16; ++i) h[i] = __ldg(B.hinvf + (size_t)i * B.M + j);
}

// y = Hbar x in FP64 for Hbar = M_A/h^2 + Kbar_A of a body with diagonal second
// moment s (Sec. 3.3): translation m/h^2; diagonal entries of A
// (s_i/h^2 + 2 V mu) x_i + V lambda (x_0 + x_4 + x_8); each transpose pair
// (A(a,i), A(i,a)) couples through V mu with masses s_i/h^2 and s_a/h^2.
__device__ __forceinline__ void hbar_apply(const double s[3], double m, double vmu, double vlam,
                                           double ih2, const double x[12], double y[12]) {
  const double tr = vlam * (x[0] + x[4] + x[8]);
  y[0] = (s[0] * ih2 + 2.0 * vmu) * x[0] + tr;
  y[4] = (s[1] * ih2 + 2.0 * vmu) * x[4] + tr;
  y[8] = (s[2] * ih2 + 2.0 * vmu) * x[8] + tr;
  // (q1 = A(1,0), q3 = A(0,1)), (q2 = A(2,0), q6 = A(0,2)), (q5 = A(2,1), q7 = A(1,2))
  y[1] = (s[0] * ih2 + vmu) * x[1] + vmu * x[3];
  y[3] = vmu * x[1] + (s[1] * ih2 + vmu) * x[3];
  y[2] = (s[0] * ih2 + vmu) * x[2] + vmu * x[6];
  y[6] = vmu * x[2] + (s[2] * ih2 + vmu) * x[6];
  y[5] = (s[1] * ih2 + vmu) * x[5] + vmu * x[7];
  y[7] = vmu * x[5] + (s[2] * ih2 + vmu) * x[7];
  const double mt = m * ih2;
  y[9] = mt * x[9];
  y[10] = mt * x[10];
  y[11] = mt * x[11];
}

// hbar_apply in double-float
__device__ __forceinline__ void hbar_apply_ff(const ff s[3], ff m, ff vmu, ff vlam, ff ih2, const ff x[12],
                                              ff y[12]) {
  const ff tr = ff_mul(vlam, ff_add(ff_add(x[0], x[4]), x[8]));
  const ff v2 = ff{2.0f * vmu.h, 2.0f * vmu.l};
  ff d[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) d[i] = ff_mul(s[i], ih2);
  y[0] = ff_fma(ff_add(d[0], v2), x[0], tr);
  y[4] = ff_fma(ff_add(d[1], v2), x[4], tr);
  y[8] = ff_fma(ff_add(d[2], v2), x[8], tr);
  y[1] = ff_fma(ff_add(d[0], vmu), x[1], ff_mul(vmu, x[3]));
  y[3] = ff_fma(vmu, x[1], ff_mul(ff_add(d[1], vmu), x[3]));
  y[2] = ff_fma(ff_add(d[0], vmu), x[2], ff_mul(vmu, x[6]));
  y[6] = ff_fma(vmu, x[2], ff_mul(ff_add(d[2], vmu), x[6]));
  y[5] = ff_fma(ff_add(d[1], vmu), x[5], ff_mul(vmu, x[7]));
  y[7] = ff_fma(vmu, x[5], ff_mul(ff_add(d[2], vmu), x[7]));
  const ff mt = ff_mul(m, ih2);
  y[9] = ff_mul(mt, x[9]);
  y[10] = ff_mul(mt, x[10]);
  y[11] = ff_mul(mt, x[11]);
}

// world displacement of rest point p under the rest-frame increment x:
// J(p) diag4(R) x = R (J(p) x)
template <typename T>
__device__ __forceinline__ void disp_at(const T R[9], const T x[12], const T p[3], T out[3]) {
  T l[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) l[a] = x[a] * p[0] + x[3 + a] * p[1] + x[6 + a] * p[2] + x[9 + a];
#pragma unroll
  for (int a = 0; a < 3; ++a) out[a] = R[3 * a] * l[0] + R[3 * a + 1] * l[1] + R[3 * a + 2] * l[2];
}

// Eq. polar in double-float: Newton's iteration X <- (X + X^{-T})/2 with
// X^{-T} = cof(X)/det(X), the same steps and stopping test as the FP64
// iteration (polar3); the first determinant is det A (det A <= 0: ST_INVERTED).
__device__ __forceinline__ int polar3_ff(const ff A[9], ff R[9], int *iters) {
  ff X[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) X[i] = A[i];
  int it = 0;
  for (; it < 40; ++it) {
    // cof(X)_rc: a b - c d as fma(a, b, -(c d))
    auto cof = [](ff a, ff b, ff c, ff d) { return ff_fma(a, b, ff_neg(ff_mul(c, d))); };
    ff C[9];
    C[0] = cof(X[4], X[8], X[5], X[7]);
    C[1] = cof(X[5], X[6], X[3], X[8]);
    C[2] = cof(X[3], X[7], X[4], X[6]);
    C[3] = cof(X[2], X[7], X[1], X[8]);
    C[4] = cof(X[0], X[8], X[2], X[6]);
    C[5] = cof(X[1], X[6], X[0], X[7]);
    C[6] = cof(X[1], X[5], X[2], X[4]);
    C[7] = cof(X[2], X[3], X[0], X[5]);
    C[8] = cof(X[0], X[4], X[1], X[3]);
    const ff d = ff_fma(X[0], C[0], ff_fma(X[1], C[1], ff_mul(X[2], C[2])));
    if (!(d.h > 0.0f)) return isfinite(d.h) ? ST_INVERTED : ST_NONFINITE;
    ff hid = ff_rcp(d);
    hid.h *= 0.5f;  // exact
    hid.l *= 0.5f;
    float diff = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const ff y = ff_fma(hid, C[i], ff{0.5f * X[i].h, 0.5f * X[i].l});
      const float dx = (y.h - X[i].h) + (y.l - X[i].l);
      diff = fmaf(dx, dx, diff);
      X[i] = y;
    }
    if (diff <= 3e-18f) break;
  }
  if (it == 40) return ST_POLAR_NOCONV;
#pragma unroll
  for (int i = 0; i < 9; ++i) R[i] = X[i];
  if (iters) *iters = it + 1;
  return 0;
}

// Eq. module1-wrench-map with the co-rotated stress of Sec. 3.3, in the rest
// frame and in double-float: fb = diag4(R^T)(M_A qdot/h + [0; m g])
// - [V vec P(R^T A); 0], P(F) = mu (F + F^T - 2I) + lambda tr(F - I) I.
// A (row-major) and R in double-float, qd the velocity, cst = (sigma_0..2,
// m, V mu, V lambda) of the body.
__device__ __forceinline__ void fbar_ff(const ff A[9], const ff R[9], const ff qd[12], const double cst[6],
                                        const StepParams &p, ff fb[12]) {
  const ff ih = ff_from(p.inv_h);
  const ff sh0 = ff_mul(ff_from(cst[0]), ih), sh1 = ff_mul(ff_from(cst[1]), ih), sh2 = ff_mul(ff_from(cst[2]), ih);
  const ff m = ff_from(cst[3]);
  const ff mh = ff_mul(m, ih);
  const ff vmu = ff_from(cst[4]), vlam = ff_from(cst[5]);
  ff fw[12];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    fw[a] = ff_mul(sh0, qd[a]);
    fw[3 + a] = ff_mul(sh1, qd[3 + a]);
    fw[6 + a] = ff_mul(sh2, qd[6 + a]);
    fw[9 + a] = ff_fma(mh, qd[9 + a], ff_mul(m, ff_from(p.g[a])));
  }
#pragma unroll
  for (int blk = 0; blk < 4; ++blk)
#pragma unroll
    for (int a = 0; a < 3; ++a)
      fb[3 * blk + a] = ff_fma(R[a], fw[3 * blk], ff_fma(R[3 + a], fw[3 * blk + 1], ff_mul(R[6 + a], fw[3 * blk + 2])));
  ff F[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      F[3 * r + c] = ff_fma(R[r], A[c], ff_fma(R[3 + r], A[3 + c], ff_mul(R[6 + r], A[6 + c])));
  const ff tr = ff_mul(vlam, ff_add(ff_add(F[0], F[4]), ff_add(F[8], ff_make(-3.0f))));
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      ff e = ff_add(F[3 * a + i], F[3 * i + a]);
      if (a == i) e = ff_add(e, ff_make(-2.0f));
      ff P = ff_mul(vmu, e);
      if (a == i) P = ff_add(P, tr);
      fb[3 * i + a] = ff_sub(fb[3 * i + a], P);
    }
}

}  // namespace mabd
