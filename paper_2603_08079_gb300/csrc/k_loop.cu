// Loop solver (Sec. 5.4, Case III, Eq. loop), FP64.  The paper splits a
// closed loop of bodies into a chain and a small block of "loop breaker"
// unknowns and solves the latter through the Schur complement of the chain.
// Here the split is made in the dual: joints 0 .. K-2 form a chain (block
// tridiagonal S_cc, factored by the chain's block cyclic reduction) and the
// last joint L = K - 1 is the breaker.  It couples to the chain's two ends:
// to joint 0 through body 0 (the corner block E = S_{0,L}) and to joint K-2
// through body K-1 (the chain coupling B[K-2] = S_{K-2,L}).  With
// S_cl = [E; 0; ...; 0; B[K-2]]:
//   (D_L - S_cl^T S_cc^{-1} S_cl) lambda_L = b_L - S_cl^T S_cc^{-1} b_c,
//   lambda_c = S_cc^{-1} (b_c - S_cl lambda_L).
// S_cc^{-1} b_c comes from the factorization pass, S_cc^{-1} S_cl from one
// right-hand-side pass per breaker row; only their values at joints 0 and
// K-2 enter the Schur complement.
#include "mabd_device.cuh"

namespace mabd {

// rhs of pass t: column t of S_cl (joint 0: E[:, t]; joint K-2: B[K-2][:, t]);
// every other entry of rb stays zero
__global__ void k_loop_column(DevChain C, int K, double *rb, int t) {
  const int r = threadIdx.x;
  if (r < 5) {
    rb[(size_t)r * K] = C.corner[5 * r + t];
    rb[(size_t)r * K + (K - 2)] = C.B[(size_t)(5 * r + t) * K + (K - 2)];
  }
}

// the solution of pass t at joints 0 and K-2 -> w[10 t .. 10 t + 9]
__global__ void k_loop_gather(int K, const double *x, double *w, int t) {
  const int r = threadIdx.x;
  if (r < 5) {
    w[10 * t + r] = x[(size_t)r * K];
    w[10 * t + 5 + r] = x[(size_t)r * K + (K - 2)];
  }
}

// The breaker's Schur complement (n = 3 or 5 rows), its multipliers into
// J.lambda, and the chain's right-hand side b_c - S_cl lambda_L into J.b
// (joints 0 and K-2).  lambda at joints 0 and K-2 holds S_cc^{-1} b_c.
__global__ void k_loop_schur(DevChain C, DevJoints J, const double *w, int *status) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const int K = J.K, L = K - 1, e = K - 2;
  const int n = J.type[L] == 0 ? 3 : 5;
  const int n0 = J.type[0] == 0 ? 3 : 5, ne = J.type[e] == 0 ? 3 : 5;
  const uint8_t fl = C.jflags[L];
  double S[5][5], bh[5];
  for (int t = 0; t < n; ++t) {
    for (int u = 0; u <= t; ++u) {
      const int i = t * (t + 1) / 2 + u;
      double d = 0.0;
      if (fl & 1) d += C.Dfirst[(size_t)i * K + L];
      if (fl & 2) d += C.Dsecond[(size_t)i * K + L];
      // - (S_cl^T S_cc^{-1} S_cl)_{tu}: column u of S_cc^{-1} S_cl at joints 0 and K-2
      for (int r = 0; r < n0; ++r) d -= C.corner[5 * r + t] * w[10 * u + r];
      for (int r = 0; r < ne; ++r) d -= C.B[(size_t)(5 * r + t) * K + e] * w[10 * u + 5 + r];
      S[t][u] = d;
    }
    double b = J.b[(size_t)t * K + L];
    for (int r = 0; r < n0; ++r) b -= C.corner[5 * r + t] * J.lambda[(size_t)r * K];
    for (int r = 0; r < ne; ++r) b -= C.B[(size_t)(5 * r + t) * K + e] * J.lambda[(size_t)r * K + e];
    bh[t] = b;
  }
  // Cholesky S = G G^T (lower), then G G^T lambda_L = bh
  bool ok = true;
  for (int c = 0; c < n; ++c) {
    double s = S[c][c];
    for (int k = 0; k < c; ++k) s -= S[c][k] * S[c][k];
    if (!(s > 0.0)) {
      ok = false;
      s = 1.0;
    }
    S[c][c] = sqrt(s);
    for (int r = c + 1; r < n; ++r) {
      double v = S[r][c];
      for (int k = 0; k < c; ++k) v -= S[r][k] * S[c][k];
      S[r][c] = v / S[c][c];
    }
  }
  if (!ok) set_status(status, ST_NOT_SPD);
  double y[5], lam[5];
  for (int i = 0; i < n; ++i) {
    double v = bh[i];
    for (int k = 0; k < i; ++k) v -= S[i][k] * y[k];
    y[i] = v / S[i][i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double v = y[i];
    for (int k = i + 1; k < n; ++k) v -= S[k][i] * lam[k];
    lam[i] = v / S[i][i];
  }
  for (int r = 0; r < 5; ++r) J.lambda[(size_t)r * K + L] = r < n ? lam[r] : 0.0;
  for (int r = 0; r < n0; ++r) {
    double v = 0.0;
    for (int t = 0; t < n; ++t) v += C.corner[5 * r + t] * lam[t];
    J.b[(size_t)r * K] -= v;
  }
  for (int r = 0; r < ne; ++r) {
    double v = 0.0;
    for (int t = 0; t < n; ++t) v += C.B[(size_t)(5 * r + t) * K + e] * lam[t];
    J.b[(size_t)r * K + e] -= v;
  }
}

void launch_loop_column(const DevChain &C, int K, double *rb, int t, cudaStream_t s) {
  k_loop_column<<<1, 32, 0, s>>>(C, K, rb, t);
}

void launch_loop_gather(int K, const double *x, double *w, int t, cudaStream_t s) {
  k_loop_gather<<<1, 32, 0, s>>>(K, x, w, t);
}

void launch_loop_schur(const DevChain &C, const DevJoints &J, const double *w, int *status, cudaStream_t s) {
  k_loop_schur<<<1, 32, 0, s>>>(C, J, w, status);
}

}  // namespace mabd
