// Structured inverse of Hbar_A = M_A/h^2 + Kbar_A (Eq. abd_final) for a body
// whose rest frame is its principal frame (diagonal second moment s), shared
// by the host set-up of mabd_prefactor and the device set-up of the
// no-allocation chain step.  Kbar_A is the Hessian in A of the small-strain
// energy V (mu |sym(A - I)|^2 + lambda/2 tr(A - I)^2) (Sec. 3.3), with
// mu = E / (2 (1 + nu)) and lambda = E nu / ((1 + nu)(1 - 2 nu)).  With the
// diagonal M_A of a principal frame, Hbar_A decouples into
//   the diagonal entries of A (q[0], q[4], q[8]): a 3x3 block with
//     s_i/h^2 + V (2 mu + lambda) on its diagonal and V lambda off it;
//   the transpose pairs (q[1], q[3]), (q[2], q[6]), (q[5], q[7]): 2x2 blocks
//     [[s_i/h^2 + V mu, V mu], [V mu, s_a/h^2 + V mu]];
//   the translation q[9..11]: (m/h^2) I3.
// Layout of the 16 entries: see HINV_N in mabd_internal.h.
#pragma once
#include <math.h>

#ifdef __CUDACC__
#define MABD_HD __host__ __device__ inline
#else
#define MABD_HD inline
#endif

namespace mabd {

// [[a, b], [b, d]]^{-1} as (d, -b, a) / det; false unless positive definite
MABD_HD bool inv2_spd(double a, double b, double d, double out[3]) {
  if (!(a > 0.0)) return false;
  const double det = a * d - b * b;
  if (!(det > 0.0)) return false;
  out[0] = d / det;
  out[1] = -b / det;
  out[2] = a / det;
  return true;
}

// false if a block is not positive definite or the result is not finite
MABD_HD bool hbar_inverse(double m, const double s[3], double V, double E, double nu, double h, double out[16]) {
  const double mu = E / (2.0 * (1.0 + nu)), lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const double ih2 = 1.0 / (h * h);
  // the 3x3 block of A's diagonal entries, inverted through its Cholesky factor
  double X[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) X[3 * r + c] = (r == c ? s[r] * ih2 + V * (2.0 * mu + lam) : V * lam);
  double L[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int c = 0; c < 3; ++c) {
    double t = X[3 * c + c];
    for (int k = 0; k < c; ++k) t -= L[3 * c + k] * L[3 * c + k];
    if (!(t > 0.0)) return false;
    L[3 * c + c] = sqrt(t);
    for (int r = c + 1; r < 3; ++r) {
      double v = X[3 * r + c];
      for (int k = 0; k < c; ++k) v -= L[3 * r + k] * L[3 * c + k];
      L[3 * r + c] = v / L[3 * c + c];
    }
  }
  double Xi[9];
  for (int c = 0; c < 3; ++c) {
    double e[3] = {0, 0, 0}, y[3], x[3];
    e[c] = 1.0;
    for (int i = 0; i < 3; ++i) {
      double v = e[i];
      for (int k = 0; k < i; ++k) v -= L[3 * i + k] * y[k];
      y[i] = v / L[3 * i + i];
    }
    for (int i = 2; i >= 0; --i) {
      double v = y[i];
      for (int k = i + 1; k < 3; ++k) v -= L[3 * k + i] * x[k];
      x[i] = v / L[3 * i + i];
    }
    for (int r = 0; r < 3; ++r) Xi[3 * r + c] = x[r];
  }
  out[0] = h * h / m;
  out[1] = Xi[0];
  out[2] = 0.5 * (Xi[1] + Xi[3]);
  out[3] = 0.5 * (Xi[2] + Xi[6]);
  out[4] = Xi[4];
  out[5] = 0.5 * (Xi[5] + Xi[7]);
  out[6] = Xi[8];
  // transpose pairs: entry (row a, column i) has mass s_i/h^2 and stiffness V mu,
  // coupled to its transpose by V mu
  const double vm = V * mu;
  if (!inv2_spd(s[0] * ih2 + vm, vm, s[1] * ih2 + vm, out + 7)) return false;   // q[1]=A(1,0), q[3]=A(0,1)
  if (!inv2_spd(s[0] * ih2 + vm, vm, s[2] * ih2 + vm, out + 10)) return false;  // q[2]=A(2,0), q[6]=A(0,2)
  if (!inv2_spd(s[1] * ih2 + vm, vm, s[2] * ih2 + vm, out + 13)) return false;  // q[5]=A(2,1), q[7]=A(1,2)
  for (int i = 0; i < 16; ++i)
    if (!isfinite(out[i])) return false;
  return out[0] > 0.0;
}

}  // namespace mabd
