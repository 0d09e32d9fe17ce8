// Host check of the principal-frame helpers (csrc/principal_frame.h): for
// random symmetric positive definite 3x3 matrices (random rotations times
// random positive diagonals, some with repeated or nearly repeated
// eigenvalues, some already diagonal) the Jacobi eigen-decomposition must
// reconstruct the matrix (1e-13 relative), give an orthonormal V with
// det V = +1, and frame_A must turn an affine part there and back exactly
// (1e-14).  Prints "failures N".
#include <cmath>
#include <cstdint>
#include <cstdio>

#include "principal_frame.h"

using namespace mabd;

static uint64_t state = 0x9e3779b97f4a7c15ULL;
static double uniform() {  // xorshift64*, in [0, 1)
  state ^= state >> 12;
  state ^= state << 25;
  state ^= state >> 27;
  return (double)((state * 0x2545f4914f6cdd1dULL) >> 11) * 0x1.0p-53;
}

static void rotation(double Q[9]) {  // from a random unit quaternion
  double q[4], n = 0.0;
  for (int i = 0; i < 4; ++i) {
    q[i] = 2.0 * uniform() - 1.0;
    n += q[i] * q[i];
  }
  n = std::sqrt(n);
  const double w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
  const double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z),     2 * (x * z + w * y),
                       2 * (x * y + w * z),     1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                       2 * (x * z - w * y),     2 * (y * z + w * x),     1 - 2 * (x * x + y * y)};
  for (int i = 0; i < 9; ++i) Q[i] = R[i];
}

int main() {
  int fail = 0;
  for (int t = 0; t < 2000; ++t) {
    double Q[9], d[3] = {0.01 + 10 * uniform(), 0.01 + 10 * uniform(), 0.01 + 10 * uniform()};
    rotation(Q);
    if (t % 7 == 0) d[1] = d[0];                   // a repeated eigenvalue
    if (t % 11 == 0) d[2] = d[0] * (1 + 1e-12);    // a nearly repeated one
    if (t % 13 == 0)
      for (int i = 0; i < 9; ++i) Q[i] = (i % 4 == 0) ? 1.0 : 0.0;  // already diagonal
    double S[3][3];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        double v = 0.0;
        for (int k = 0; k < 3; ++k) v += Q[3 * r + k] * d[k] * Q[3 * c + k];
        S[r][c] = v;
      }
    const double S6[6] = {S[0][0], S[1][1], S[2][2], S[0][1], S[0][2], S[1][2]};
    double w[3], V[9];
    if (!sym3_eigen(S6, w, V)) {
      ++fail;
      std::printf("case %d: no convergence\n", t);
      continue;
    }
    double scale = 0.0, err = 0.0, orth = 0.0;
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        double v = 0.0, o = 0.0;
        for (int k = 0; k < 3; ++k) {
          v += V[3 * r + k] * w[k] * V[3 * c + k];
          o += V[3 * k + r] * V[3 * k + c];
        }
        scale = std::fmax(scale, std::fabs(S[r][c]));
        err = std::fmax(err, std::fabs(v - S[r][c]));
        orth = std::fmax(orth, std::fabs(o - (r == c ? 1.0 : 0.0)));
      }
    const double det = V[0] * (V[4] * V[8] - V[5] * V[7]) - V[1] * (V[3] * V[8] - V[5] * V[6]) +
                       V[2] * (V[3] * V[7] - V[4] * V[6]);
    if (!(err <= 1e-13 * scale) || !(orth <= 1e-13) || !(std::fabs(det - 1.0) <= 1e-13)) {
      ++fail;
      std::printf("case %d: reconstruction %.3g, orthonormality %.3g, det %.17g\n", t, err / scale, orth, det);
    }
    double x[12], y[12], z[12];
    for (int i = 0; i < 12; ++i) x[i] = 2.0 * uniform() - 1.0;
    frame_A(x, V, false, y);
    frame_A(y, V, true, z);
    double e = 0.0;
    for (int i = 0; i < 12; ++i) e = std::fmax(e, std::fabs(z[i] - x[i]));
    for (int i = 9; i < 12; ++i) e = std::fmax(e, std::fabs(y[i] - x[i]));
    if (!(e <= 1e-14)) {
      ++fail;
      std::printf("case %d: frame round trip %.3g\n", t, e);
    }
  }
  std::printf("failures %d\n", fail);
  return fail ? 1 : 0;
}
