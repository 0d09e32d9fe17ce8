// Principal frames of bodies given with a non-diagonal second moment (host
// code, no CUDA): the eigen-decomposition Sigma = V diag(w) V^T and the
// change of a 12-vector's affine part between the caller's rest frame and
// the principal one (A_principal = A V).
#pragma once
#include <cmath>

namespace mabd {

// Eigen-decomposition of a symmetric 3x3 matrix (second moment xx, yy, zz,
// xy, xz, yz) by cyclic Jacobi rotations (Jacobi's method; Golub and Van
// Loan, Matrix Computations, Sec. 8.5): S = V diag(w) V^T with V a rotation
// (row-major, columns the principal axes, det +1).
inline bool sym3_eigen(const double S6[6], double w[3], double V[9]) {
  double a[3][3] = {{S6[0], S6[3], S6[4]}, {S6[3], S6[1], S6[5]}, {S6[4], S6[5], S6[2]}};
  double v[3][3] = {{1.0, 0.0, 0.0}, {0.0, 1.0, 0.0}, {0.0, 0.0, 1.0}};
  bool done = false;
  for (int sweep = 0; sweep < 64 && !done; ++sweep) {
    const double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
    const double dia = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
    // converged when the off-diagonal entries are at rounding level of the
    // diagonal (relative 1e-15)
    if (off <= 1e-30 * dia) {
      done = true;
      break;
    }
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (a[p][q] == 0.0) continue;
        // the rotation in the (p, q) plane that zeroes a[p][q]
        const double th = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
        const double t = (th >= 0.0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < 3; ++k) {
          const double x = a[k][p], y = a[k][q];
          a[k][p] = c * x - sn * y;
          a[k][q] = sn * x + c * y;
        }
        for (int k = 0; k < 3; ++k) {
          const double x = a[p][k], y = a[q][k];
          a[p][k] = c * x - sn * y;
          a[q][k] = sn * x + c * y;
        }
        for (int k = 0; k < 3; ++k) {
          const double x = v[k][p], y = v[k][q];
          v[k][p] = c * x - sn * y;
          v[k][q] = sn * x + c * y;
        }
      }
  }
  if (!done) return false;
  const double det = v[0][0] * (v[1][1] * v[2][2] - v[1][2] * v[2][1]) -
                     v[0][1] * (v[1][0] * v[2][2] - v[1][2] * v[2][0]) +
                     v[0][2] * (v[1][0] * v[2][1] - v[1][1] * v[2][0]);
  if (det < 0.0)
    for (int k = 0; k < 3; ++k) v[k][2] = -v[k][2];
  for (int r = 0; r < 3; ++r) {
    w[r] = a[r][r];
    for (int c = 0; c < 3; ++c) V[3 * r + c] = v[r][c];
  }
  return true;
}

// the affine part of a 12-vector (A(r, c) = x[3c + r]) times V (back = false)
// or V^T (back = true); the translation is copied
inline void frame_A(const double x[12], const double V[9], bool back, double y[12]) {
  double t[12];
  for (int c = 0; c < 3; ++c)
    for (int r = 0; r < 3; ++r) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += x[3 * k + r] * (back ? V[3 * c + k] : V[3 * k + c]);
      t[3 * c + r] = acc;
    }
  for (int i = 0; i < 9; ++i) y[i] = t[i];
  for (int i = 9; i < 12; ++i) y[i] = x[i];
}

}  // namespace mabd
