// Tree path of one M-ABD step (FP64), Sec. 5.3 (Alg. 2, Eq. module3-kkt),
// read as the exact constraint-row elimination in body space:
//   upward (deepest level first), body j with parent joint rows G (on j) and
//   P (on the parent):
//     Hhat_j = Hbar_j + sum_children U_i U_i^T,  fhat_j = fbar_j - sum_children v_i
//     y = Hhat_j^{-1} fhat_j, X = Hhat_j^{-1} G^T, D = G X = L_D L_D^T,
//     e = G y + C(q_n),  U = P^T L_D^{-T},  v = P^T D^{-1} e   (to the parent)
//   downward (roots first):
//     lambda = D^{-1}(e + P dq_parent),  dq_j = y - X lambda.
// Everything of body j is kept in its rest frame (rows s [p;1] (x) R_j^T d),
// so a leaf uses the structured Hbar^{-1}; bodies with children factor their
// dense 12x12 Hhat (packed lower storage).
#include "mabd_device.cuh"

namespace mabd {

__device__ __forceinline__ int p12(int r, int c) { return r * (r + 1) / 2 + c; }  // r >= c

// dense Hbar (packed lower, 78) from the body constants (Eq. abd_final)
__device__ __forceinline__ void hbar_dense(const DevBodies &B, int j, double ih2, double H[78]) {
  const int M = B.M;
  const double s[3] = {ldg(B.sig + j), ldg(B.sig + M + j), ldg(B.sig + 2 * (size_t)M + j)};
  const double vm = ldg(B.vmu + j), vl = ldg(B.vlam + j), m = ldg(B.mass + j);
#pragma unroll
  for (int i = 0; i < 78; ++i) H[i] = 0.0;
  // diagonal entries of A: q[0], q[4], q[8]
  const int dg[3] = {0, 4, 8};
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b <= a; ++b) H[p12(dg[a], dg[b])] = a == b ? s[a] * ih2 + 2.0 * vm + vl : vl;
  // transpose pairs (first index has column i, second column k)
  const int pa[3] = {1, 2, 5}, pb[3] = {3, 6, 7};
  const int ca[3] = {0, 0, 1}, cb[3] = {1, 2, 2};
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    H[p12(pa[t], pa[t])] = s[ca[t]] * ih2 + vm;
    H[p12(pb[t], pb[t])] = s[cb[t]] * ih2 + vm;
    H[p12(pb[t], pa[t])] = vm;
  }
#pragma unroll
  for (int a = 9; a < 12; ++a) H[p12(a, a)] = m * ih2;
}

__device__ __forceinline__ void hbar_mul(const double H[78], const double x[12], double y[12]) {
#pragma unroll
  for (int r = 0; r < 12; ++r) {
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 12; ++c) s += H[r >= c ? p12(r, c) : p12(c, r)] * x[c];
    y[r] = s;
  }
}

__device__ __forceinline__ bool chol12(double A[78]) {  // in place
  bool ok = true;
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    double s = A[p12(c, c)];
#pragma unroll
    for (int k = 0; k < c; ++k) s -= A[p12(c, k)] * A[p12(c, k)];
    if (!(s > 0.0)) {
      ok = false;
      s = 1.0;
    }
    const double d = sqrt(s), id = 1.0 / d;
    A[p12(c, c)] = d;
#pragma unroll
    for (int r = c + 1; r < 12; ++r) {
      double t = A[p12(r, c)];
#pragma unroll
      for (int k = 0; k < c; ++k) t -= A[p12(r, k)] * A[p12(c, k)];
      A[p12(r, c)] = t * id;
    }
  }
  return ok;
}

__device__ __forceinline__ void chol12_solve(const double L[78], const double b[12], double x[12]) {
  double y[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    double s = b[i];
#pragma unroll
    for (int k = 0; k < i; ++k) s -= L[p12(i, k)] * y[k];
    y[i] = s / L[p12(i, i)];
  }
#pragma unroll
  for (int i = 11; i >= 0; --i) {
    double s = y[i];
#pragma unroll
    for (int k = i + 1; k < 12; ++k) s -= L[p12(k, i)] * x[k];
    x[i] = s / L[p12(i, i)];
  }
}

// small dense Cholesky (n <= 10, packed lower)
template <int NMAX>
__device__ __forceinline__ bool chol_small(double A[NMAX * (NMAX + 1) / 2], int n) {
  bool ok = true;
  for (int c = 0; c < n; ++c) {
    double s = A[p12(c, c)];
    for (int k = 0; k < c; ++k) s -= A[p12(c, k)] * A[p12(c, k)];
    if (!(s > 0.0)) {
      ok = false;
      s = 1.0;
    }
    const double d = sqrt(s), id = 1.0 / d;
    A[p12(c, c)] = d;
    for (int r = c + 1; r < n; ++r) {
      double t = A[p12(r, c)];
      for (int k = 0; k < c; ++k) t -= A[p12(r, k)] * A[p12(c, k)];
      A[p12(r, c)] = t * id;
    }
  }
  return ok;
}

__device__ __forceinline__ void lsolve_small(const double *L, int n, const double *b, double *x) {
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[p12(i, k)] * x[k];
    x[i] = s / L[p12(i, i)];
  }
}

__device__ __forceinline__ void ltsolve_small(const double *L, int n, const double *b, double *x) {
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int k = i + 1; k < n; ++k) s -= L[p12(k, i)] * x[k];
    x[i] = s / L[p12(i, i)];
  }
}

constexpr int RMAX = 10;  // rows eliminated at a root (two one-sided joints)

__global__ void __launch_bounds__(64) k_tree_up(DevBodies B, DevJoints J, DevTree T, int lo, int hi,
                                                StepParams p, int *status) {
  const int j = lo + blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= hi) return;
  const int M = B.M, K = J.K;
  double R[9], h[16];
  load_R(B.R, M, j, R);
  load_hinv(B, j, h);
  const int nch = T.ccount[j];
  double L[78];
  double y[12];
  if (nch == 0) {
    load12(B.ubar, M, j, y);
  } else {
    const double ih2 = p.inv_h * p.inv_h;
    hbar_dense(B, j, ih2, L);
    double ub[12], f[12];
    load12(B.ubar, M, j, ub);
    hbar_mul(L, ub, f);  // fbar = Hbar ubar
    const int c0 = T.cfirst[j];
    for (int c = c0; c < c0 + nch; ++c) {
#pragma unroll
      for (int a = 0; a < 12; ++a) f[a] -= T.v[(size_t)a * M + c];
      const int Cc = J.type[T.pjoint[c]] == 0 ? 3 : 5;
      for (int t = 0; t < Cc; ++t) {
        double u[12];
#pragma unroll
        for (int a = 0; a < 12; ++a) u[a] = T.U[(size_t)(5 * a + t) * M + c];
#pragma unroll
        for (int r = 0; r < 12; ++r)
#pragma unroll
          for (int cc = 0; cc <= r; ++cc) L[p12(r, cc)] += u[r] * u[cc];
      }
    }
    if (!chol12(L)) set_status(status, ST_NOT_SPD);
    chol12_solve(L, f, y);
  }
  // rows eliminated here: the parent joint, or a root's one-sided joints
  const int par = T.parent[j];
  const int rid = T.root_id[j];
  double E[RMAX][3], P[4][3];
  int pt[RMAX], ks[2] = {-1, -1}, cs[2] = {0, 0};
  int n = 0;
  if (par >= 0) {
    ks[0] = T.pjoint[j];
    double E5[5][3], P2[2][3];
    int pt5[5];
    cs[0] = joint_rows_rest(J, ks[0], T.pside[j], R, E5, P2, pt5);
    for (int r = 0; r < cs[0]; ++r) {
      E[r][0] = E5[r][0]; E[r][1] = E5[r][1]; E[r][2] = E5[r][2];
      pt[r] = pt5[r];
    }
    P[0][0] = P2[0][0]; P[0][1] = P2[0][1]; P[0][2] = P2[0][2];
    P[1][0] = P2[1][0]; P[1][1] = P2[1][1]; P[1][2] = P2[1][2];
    n = cs[0];
  } else if (rid >= 0) {
    for (int w = 0; w < 2; ++w) {
      const int k = T.root_joint[(size_t)w * T.nroots + rid];
      if (k < 0) continue;
      double E5[5][3], P2[2][3];
      int pt5[5];
      ks[w] = k;
      cs[w] = joint_rows_rest(J, k, T.root_side[(size_t)w * T.nroots + rid], R, E5, P2, pt5);
      for (int r = 0; r < cs[w]; ++r) {
        E[n + r][0] = E5[r][0]; E[n + r][1] = E5[r][1]; E[n + r][2] = E5[r][2];
        pt[n + r] = 2 * w + pt5[r];
      }
      for (int a = 0; a < 3; ++a) {
        P[2 * w][a] = P2[0][a];
        P[2 * w + 1][a] = P2[1][a];
      }
      n += cs[w];
    }
  }
  // X = Hhat^{-1} G^T, D = G X, e = G y + C
  double X[RMAX][12];
  double D[RMAX * (RMAX + 1) / 2];
  double e[RMAX];
  const double rr = p.residual_rhs ? 1.0 : 0.0;
  for (int r = 0; r < n; ++r) {
    double w[12];
    kron_row(P[pt[r]], E[r], w);
    if (nch == 0) hinv_apply(h, w, X[r]);
    else chol12_solve(L, w, X[r]);
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 12; ++a) s += w[a] * y[a];
    const int k = r < cs[0] ? ks[0] : ks[1];
    const int rl = r < cs[0] ? r : r - cs[0];
    e[r] = s + rr * J.c[(size_t)rl * K + k];
    for (int t = 0; t <= r; ++t) {
      double d = 0.0;
#pragma unroll
      for (int a = 0; a < 12; ++a) d += w[a] * X[t][a];
      D[p12(r, t)] = d;
    }
  }
  if (n > 0 && !chol_small<RMAX>(D, n)) set_status(status, ST_NOT_SPD);
  if (par >= 0) {
#pragma unroll
    for (int a = 0; a < 12; ++a) {
#pragma unroll
      for (int r = 0; r < 5; ++r) T.X[(size_t)(5 * a + r) * M + j] = r < n ? X[r][a] : 0.0;
      T.y[(size_t)a * M + j] = y[a];
    }
    for (int i = 0; i < 15; ++i) T.LD[(size_t)i * M + j] = i < n * (n + 1) / 2 ? D[i] : 0.0;
    for (int r = 0; r < 5; ++r) T.e[(size_t)r * M + j] = r < n ? e[r] : 0.0;
    // contribution to the parent, in the parent's rest frame
    double Rp[9], Ep[5][3], Pp[2][3];
    int ptp[5];
    load_R(B.R, M, par, Rp);
    joint_rows_rest(J, ks[0], 1 - T.pside[j], Rp, Ep, Pp, ptp);
    double wl[5];
    lsolve_small(D, n, e, wl);
    // Z = L_D^{-1} Pbar (n x 12), column by column
    double Z[5][12];
#pragma unroll
    for (int a = 0; a < 12; ++a) {
      double col[5], z[5];
      for (int r = 0; r < n; ++r) {
        double w[12];
        kron_row(Pp[ptp[r]], Ep[r], w);
        col[r] = w[a];
      }
      lsolve_small(D, n, col, z);
      for (int r = 0; r < n; ++r) Z[r][a] = z[r];
    }
#pragma unroll
    for (int a = 0; a < 12; ++a) {
      double vv = 0.0;
      for (int r = 0; r < 5; ++r) {
        const double u = r < n ? Z[r][a] : 0.0;
        T.U[(size_t)(5 * a + r) * M + j] = u;
        vv += u * (r < n ? wl[r] : 0.0);
      }
      T.v[(size_t)a * M + j] = vv;
    }
  } else {
    const int nr = T.nroots;
#pragma unroll
    for (int a = 0; a < 12; ++a) {
      for (int r = 0; r < RMAX; ++r) T.rX[(size_t)(RMAX * a + r) * nr + rid] = r < n ? X[r][a] : 0.0;
      T.y[(size_t)a * M + j] = y[a];
    }
    for (int i = 0; i < RMAX * (RMAX + 1) / 2; ++i)
      T.rLD[(size_t)i * nr + rid] = i < n * (n + 1) / 2 ? D[i] : 0.0;
    for (int r = 0; r < RMAX; ++r) T.re[(size_t)r * nr + rid] = r < n ? e[r] : 0.0;
  }
}

__global__ void __launch_bounds__(128) k_tree_down(DevBodies B, DevJoints J, DevTree T, int lo,
                                                   int hi, StepParams p) {
  const int j = lo + blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= hi) return;
  const int M = B.M, K = J.K;
  const int par = T.parent[j];
  double dqb[12];
  double y[12];
  load12(T.y, M, j, y);
  if (par >= 0) {
    const int k = T.pjoint[j];
    const int type = J.type[k];
    const int n = type == 0 ? 3 : 5;
    const int pside = 1 - T.pside[j];
    // P dq_parent: rows s_p d_r^T J(p_r) dq_p in the world frame
    double dqp[12];
    load12(T.dq, M, par, dqp);
    double pts[2][3];
    load3(pside == 0 ? J.pa1 : J.pb1, K, k, pts[0]);
    if (type == 1) load3(pside == 0 ? J.pa2 : J.pb2, K, k, pts[1]);
    double x[2][3];
    for (int q = 0; q < 1 + type; ++q)
#pragma unroll
      for (int a = 0; a < 3; ++a)
        x[q][a] = dqp[a] * pts[q][0] + dqp[3 + a] * pts[q][1] + dqp[6 + a] * pts[q][2] + dqp[9 + a];
    double RH[9];
    if (type == 1) load_R(J.RH, K, k, RH);
    const double sp = pside == 0 ? 1.0 : -1.0;
    double rhs[5], lam[5], t[5], LD[15];
    for (int r = 0; r < n; ++r) {
      double d[3];
      row_dir(type, RH, r, d);
      const int q = r < 3 ? 0 : 1;
      rhs[r] = T.e[(size_t)r * M + j] + sp * (d[0] * x[q][0] + d[1] * x[q][1] + d[2] * x[q][2]);
    }
    for (int i = 0; i < n * (n + 1) / 2; ++i) LD[i] = T.LD[(size_t)i * M + j];
    lsolve_small(LD, n, rhs, t);
    ltsolve_small(LD, n, t, lam);
    for (int r = 0; r < n; ++r) J.lambda[(size_t)r * K + k] = lam[r];
#pragma unroll
    for (int a = 0; a < 12; ++a) {
      double s = y[a];
      for (int r = 0; r < n; ++r) s -= T.X[(size_t)(5 * a + r) * M + j] * lam[r];
      dqb[a] = s;
    }
  } else {
    const int rid = T.root_id[j];
    const int nr = T.nroots;
    int n = 0, cs[2] = {0, 0}, ks[2] = {-1, -1};
    for (int w = 0; w < 2; ++w) {
      ks[w] = rid >= 0 ? T.root_joint[(size_t)w * nr + rid] : -1;
      cs[w] = ks[w] < 0 ? 0 : (J.type[ks[w]] == 0 ? 3 : 5);
      n += cs[w];
    }
    double lam[RMAX], t[RMAX], e[RMAX], LD[RMAX * (RMAX + 1) / 2];
    for (int r = 0; r < n; ++r) e[r] = T.re[(size_t)r * nr + rid];
    for (int i = 0; i < n * (n + 1) / 2; ++i) LD[i] = T.rLD[(size_t)i * nr + rid];
    if (n > 0) {
      lsolve_small(LD, n, e, t);
      ltsolve_small(LD, n, t, lam);
    }
    for (int r = 0; r < n; ++r) {
      const int w = r < cs[0] ? 0 : 1;
      J.lambda[(size_t)(r - (w ? cs[0] : 0)) * K + ks[w]] = lam[r];
    }
#pragma unroll
    for (int a = 0; a < 12; ++a) {
      double s = y[a];
      for (int r = 0; r < n; ++r) s -= T.rX[(size_t)(RMAX * a + r) * nr + rid] * lam[r];
      dqb[a] = s;
    }
  }
  double R[9];
  load_R(B.R, M, j, R);
#pragma unroll
  for (int blk = 0; blk < 4; ++blk) {
    double dq[3];
    mv3(R, dqb + 3 * blk, dq);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const size_t o = (size_t)(3 * blk + a) * M + j;
      T.dq[o] = dq[a];
      B.q[o] += dq[a];
      B.qd[o] = dq[a] * p.inv_h;
    }
  }
}

void launch_tree_up(const DevBodies &B, const DevJoints &J, const DevTree &T, int lo, int hi,
                    const StepParams &p, int *status, cudaStream_t s) {
  const int n = hi - lo;
  if (n > 0) k_tree_up<<<(n + 63) / 64, 64, 0, s>>>(B, J, T, lo, hi, p, status);
}

void launch_tree_down(const DevBodies &B, const DevJoints &J, const DevTree &T, int lo, int hi,
                      const StepParams &p, int * /*status*/, cudaStream_t s) {
  const int n = hi - lo;
  if (n > 0) k_tree_down<<<(n + 127) / 128, 128, 0, s>>>(B, J, T, lo, hi, p);
}

}  // namespace mabd
