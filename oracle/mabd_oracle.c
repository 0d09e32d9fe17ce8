/*
 * CPU FP64 oracle for one M-ABD time step -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test-suite, the package smoke check and the benchmark's CPU
 * baseline may load this library.  It is plain, slow, single-threaded C
 * written from M-ABD (arXiv 2603.08079):
 *   Sec. 3.1 Eq. abd / abd_dof     x = A xbar + t = J(xbar) q
 *   Sec. 3.2 Eq. newton_abd         H_A = M_A / h^2 + K_A
 *   Sec. 3.3 Eq. polar, reduced_K   R = A (A^T A)^(-1/2),  K_A = diag4(R) Kbar_A diag4(R^T)
 *   Sec. 3.3 (linear elasticity)    dPsi/dA = mu (A + A^T - 2I) + lambda tr(A - I) I,
 *                                   applied co-rotated as R P(R^T A)
 *   Sec. 3.4 Eq. abd_final          Hbar_A diag4(R^T) dq = diag4(R^T) f_A, Hbar_A prefactored
 *   Sec. 4.2 Eq. ball, 4.3 Eq. hinge, Sec. 5.1 Eq. pcpq (frozen joint frame)
 *   Sec. 5 Eq. kkt (with the footnote's -C(q_n) rhs), Eq. primal, Eq. dual
 *   Sec. 5.2 Eq. chain-Schur-blocks, chain-b, chain-btd (block Thomas)
 *   Sec. 5.3 Alg. 2 / Eq. module3-kkt read as exact constraint-row Schur
 *            elimination in body space (leaf-to-root, then root-to-leaf)
 *   Sec. 5.5 graph: block-Jacobi preconditioned CG on the dual matrix
 *   Sec. 5.2 Eq. recover-dq-explicit  dq_j = H_j^{-1}(f_j - sum_k G_kj^T lambda_k)
 * Variants (scene flags): Alg. 1 / Eq. len_preserving for the unconstrained
 * solve (rotation_mode 1); the full constraint gradient of Eq.
 * constraint_gradient / pcpr / r_gradient (jacobian_mode 1).
 * No blocking, fusion or reordering beyond the definitions.
 */
#include "mabd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define IDX12(r, c) ((r) * 12 + (c))

/* ------------------------------------------------------------------ */
/* 3x3 helpers (row-major)                                             */
/* ------------------------------------------------------------------ */
static double det3(const double A[9]) {
  return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
         A[2] * (A[3] * A[7] - A[4] * A[6]);
}

static int inv3(const double A[9], double B[9]) {
  double d = det3(A);
  if (d == 0.0 || !isfinite(d)) return 1;
  B[0] = (A[4] * A[8] - A[5] * A[7]) / d;
  B[1] = (A[2] * A[7] - A[1] * A[8]) / d;
  B[2] = (A[1] * A[5] - A[2] * A[4]) / d;
  B[3] = (A[5] * A[6] - A[3] * A[8]) / d;
  B[4] = (A[0] * A[8] - A[2] * A[6]) / d;
  B[5] = (A[2] * A[3] - A[0] * A[5]) / d;
  B[6] = (A[3] * A[7] - A[4] * A[6]) / d;
  B[7] = (A[1] * A[6] - A[0] * A[7]) / d;
  B[8] = (A[0] * A[4] - A[1] * A[3]) / d;
  return 0;
}

static void mm3(const double A[9], const double B[9], double C[9]) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[3 * r + k] * B[3 * k + c];
      C[3 * r + c] = s;
    }
}

static void mtm3(const double A[9], const double B[9], double C[9]) { /* A^T B */
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[3 * k + r] * B[3 * k + c];
      C[3 * r + c] = s;
    }
}

static void mv3(const double A[9], const double x[3], double y[3]) {
  for (int r = 0; r < 3; ++r) y[r] = A[3 * r] * x[0] + A[3 * r + 1] * x[1] + A[3 * r + 2] * x[2];
}

static void mtv3(const double A[9], const double x[3], double y[3]) {
  for (int r = 0; r < 3; ++r) y[r] = A[r] * x[0] + A[3 + r] * x[1] + A[6 + r] * x[2];
}

static void A_of_q(const double *q, double A[9]) { /* A(r,c) = q[3c+r] */
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) A[3 * r + c] = q[3 * c + r];
}

/* x_alpha(pa) - x_beta(pb) with x(p) = A p + t (Eq. abd_dof, Eq. ball), grouped as (A_a pa - A_b pb) + (t_a - t_b)
   so that assemblies far from the origin keep the gap to round-off of the
   body size rather than of the absolute coordinates; qb == NULL: pb is a
   world point. */
static void gap_of(const double *qa, const double pa[3], const double *qb, const double pb[3],
                   double d[3]) {
  for (int a = 0; a < 3; ++a) {
    double la = qa[a] * pa[0] + qa[3 + a] * pa[1] + qa[6 + a] * pa[2];
    if (qb) {
      double lb = qb[a] * pb[0] + qb[3 + a] * pb[1] + qb[6 + a] * pb[2];
      d[a] = (la - lb) + (qa[9 + a] - qb[9 + a]);
    } else {
      d[a] = la + (qa[9 + a] - pb[a]);
    }
  }
}

static void normalize3(const double a[3], double b[3]) {
  double n = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  b[0] = a[0] / n;
  b[1] = a[1] / n;
  b[2] = a[2] / n;
}

/* ------------------------------------------------------------------ */
/* Sec. 3.2: generalized mass, Sec. 3.3: rest-shape stiffness          */
/* ------------------------------------------------------------------ */
static void sigma4(double m, const double S[6], double Sg[16]) {
  /* Sigma_hat = [[Sigma, 0],[0, m]] (4x4): block (i,j) of M_A is Sigma_hat_ij I3 */
  memset(Sg, 0, 16 * sizeof(double));
  Sg[0] = S[0]; Sg[5] = S[1]; Sg[10] = S[2];
  Sg[1] = Sg[4] = S[3];
  Sg[2] = Sg[8] = S[4];
  Sg[6] = Sg[9] = S[5];
  Sg[15] = m;
}

int ora_mass_matrix(double m, const double S[6], double MA[144]) {
  double Sg[16];
  sigma4(m, S, Sg);
  memset(MA, 0, 144 * sizeof(double));
  for (int bi = 0; bi < 4; ++bi)
    for (int bj = 0; bj < 4; ++bj)
      for (int a = 0; a < 3; ++a) MA[IDX12(3 * bi + a, 3 * bj + a)] = Sg[4 * bi + bj];
  return ORA_OK;
}

static void lame(double E, double nu, double *mu, double *lam) {
  *mu = E / (2.0 * (1.0 + nu));
  *lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
}

/* Hessian of V * Psi with Psi = mu |sym(A) - I|^2 + lambda/2 tr(A - I)^2,
   whose gradient is the linear-elastic stress of Sec. 3.3:
   d vec(P) / d vec(A) = mu (I9 + K33) + lambda vec(I) vec(I)^T, zero on t. */
int ora_stiffness_matrix(double V, double E, double nu, double KA[144]) {
  double mu, lam;
  lame(E, nu, &mu, &lam);
  memset(KA, 0, 144 * sizeof(double));
  for (int i = 0; i < 3; ++i)
    for (int a = 0; a < 3; ++a)
      for (int j = 0; j < 3; ++j)
        for (int b = 0; b < 3; ++b) {
          double v = mu * ((i == j && a == b) ? 1.0 : 0.0) +
                     mu * ((a == j && b == i) ? 1.0 : 0.0) +
                     lam * ((a == i && b == j) ? 1.0 : 0.0);
          KA[IDX12(3 * i + a, 3 * j + b)] = V * v;
        }
  return ORA_OK;
}

/* Eq. abd_final: Hbar_A = M_A / h^2 + Kbar_A */
int ora_system_matrix(double m, const double S[6], double V, double E, double nu,
                      double h, double H[144]) {
  double MA[144], KA[144];
  ora_mass_matrix(m, S, MA);
  ora_stiffness_matrix(V, E, nu, KA);
  for (int i = 0; i < 144; ++i) H[i] = MA[i] / (h * h) + KA[i];
  return ORA_OK;
}

/* ------------------------------------------------------------------ */
/* dense Cholesky (general n, row-major, lower)                         */
/* ------------------------------------------------------------------ */
static int cholesky(int n, const double *A, double *L) {
  memset(L, 0, (size_t)n * n * sizeof(double));
  for (int j = 0; j < n; ++j) {
    double s = A[j * n + j];
    for (int k = 0; k < j; ++k) s -= L[j * n + k] * L[j * n + k];
    if (!(s > 0.0)) return ORA_ERR_NOT_SPD;
    double d = sqrt(s);
    L[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = A[i * n + j];
      for (int k = 0; k < j; ++k) t -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = t / d;
    }
  }
  return ORA_OK;
}

static void chol_solve(int n, const double *L, const double *b, double *x) {
  double *y = (double *)malloc(sizeof(double) * n);
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[i * n + k] * y[k];
    y[i] = s / L[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
    x[i] = s / L[i * n + i];
  }
  free(y);
}

static void lower_solve(int n, const double *L, const double *b, double *y) {
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[i * n + k] * y[k];
    y[i] = s / L[i * n + i];
  }
}

int ora_cholesky12(const double A[144], double L[144]) { return cholesky(12, A, L); }

/* ------------------------------------------------------------------ */
/* Eq. polar: R = A (A^T A)^(-1/2) by Higham's Newton iteration         */
/* X <- (X + X^{-T}) / 2 from X = A                                    */
/* ------------------------------------------------------------------ */
int ora_polar(const double A[9], double R[9], int32_t *iters) {
  for (int i = 0; i < 9; ++i)
    if (!isfinite(A[i])) return ORA_ERR_NONFINITE;
  if (!(det3(A) > 0.0)) return ORA_ERR_INVERTED;
  double X[9], Xi[9], Y[9];
  memcpy(X, A, sizeof(X));
  int it;
  double diff = 0.0, nrm = 1.0;
  for (it = 1; it <= 100; ++it) {
    if (inv3(X, Xi)) return ORA_ERR_INVERTED;
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) Y[3 * r + c] = 0.5 * (X[3 * r + c] + Xi[3 * c + r]);
    diff = 0.0;
    nrm = 0.0;
    for (int i = 0; i < 9; ++i) {
      diff += (Y[i] - X[i]) * (Y[i] - X[i]);
      nrm += Y[i] * Y[i];
    }
    memcpy(X, Y, sizeof(X));
    if (sqrt(diff) <= 1e-15 * sqrt(nrm)) break;
  }
  if (iters) *iters = it;
  if (it > 100 && sqrt(diff) > 1e-12 * sqrt(nrm)) return ORA_ERR_NO_CONV;
  memcpy(R, X, sizeof(X));
  return ORA_OK;
}

/* Sec. 3.3 linear elasticity: P(F) = mu (F + F^T - 2I) + lambda tr(F - I) I */
void ora_elastic_stress(const double F[9], double mu, double lam, double P[9]) {
  double tr = F[0] + F[4] + F[8] - 3.0;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      P[3 * r + c] = mu * (F[3 * r + c] + F[3 * c + r] - 2.0 * (r == c)) + lam * tr * (r == c);
}

/* Right-hand side of Eq. newton_abd for one Newton step started at x = x_n
   with implicit Euler (Eq. variation_energy):
     f = M_A qdot / h + f_ext,A - V vec(R P(R^T A))     (world frame)
   f_ext,A = G^T W_ext = [0_9; m g] for gravity at the COM (Eq. module1-wrench-map). */
int ora_body_rhs(const ora_scene *sc, int64_t j, const double *q, const double *qd,
                 double f[12], double R[9]) {
  const double *qj = q + 12 * j, *qdj = qd + 12 * j;
  double A[9], F[9], P[9], RP[9], Sg[16], mu, lam;
  A_of_q(qj, A);
  int st = ora_polar(A, R, NULL);
  if (st) return st;
  lame(sc->young[j], sc->poisson[j], &mu, &lam);
  mtm3(R, A, F);
  ora_elastic_stress(F, mu, lam, P);
  mm3(R, P, RP);
  sigma4(sc->mass[j], sc->second_moment + 6 * j, Sg);
  double h = sc->h, V = sc->volume[j];
  for (int i = 0; i < 4; ++i)
    for (int a = 0; a < 3; ++a) {
      double s = 0.0;
      for (int bj = 0; bj < 4; ++bj) s += Sg[4 * i + bj] * qdj[3 * bj + a];
      f[3 * i + a] = s / h;
    }
  for (int i = 0; i < 3; ++i)
    for (int a = 0; a < 3; ++a) f[3 * i + a] -= V * RP[3 * a + i];
  for (int a = 0; a < 3; ++a) f[9 + a] += sc->mass[j] * sc->g[a];
  return ORA_OK;
}

/* Sec. 4.3: R_H = I + [v]x + [v]x^2 / (1 + a_y),  v = a x e_y  (R_H a = e_y) */
void ora_hinge_frame(const double a[3], double RH[9]) {
  double v[3] = {-a[2], 0.0, a[0]};
  double Vx[9] = {0.0, -v[2], v[1], v[2], 0.0, -v[0], -v[1], v[0], 0.0};
  double V2[9];
  mm3(Vx, Vx, V2);
  for (int i = 0; i < 9; ++i) RH[i] = (i % 4 == 0 ? 1.0 : 0.0) + Vx[i] + V2[i] / (1.0 + a[1]);
}

/* Alg. 1 (Sec. 3.4): the unconstrained solve of one body with each
   rotation of a 3-block replaced by the length-preserving map of Eq.
   len_preserving.  The four blocks f_k of f are taken to the rest frame as
   A^T f_k rescaled to |f_k|, Hbar_A dp = f~ is solved with the prefactored
   L, and each block dp_k is taken back as A dp_k rescaled to |dp_k|.  A
   zero block stays zero (the rescaling is bounded; its limit is 0). */
void ora_alg1_solve(const double L[144], const double A[9], const double f[12], double u[12]) {
  double ft[12], dp[12];
  for (int k = 0; k < 4; ++k) {
    const double *fk = f + 3 * k;
    double *t = ft + 3 * k;
    const double l2 = fk[0] * fk[0] + fk[1] * fk[1] + fk[2] * fk[2];
    mtv3(A, fk, t);
    const double n2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    const double s = n2 > 0.0 ? sqrt(l2 / n2) : 0.0;
    for (int a = 0; a < 3; ++a) t[a] *= s;
  }
  chol_solve(12, L, ft, dp);
  for (int k = 0; k < 4; ++k) {
    const double *pk = dp + 3 * k;
    double *t = u + 3 * k;
    const double l2 = pk[0] * pk[0] + pk[1] * pk[1] + pk[2] * pk[2];
    mv3(A, pk, t);
    const double n2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    const double s = n2 > 0.0 ? sqrt(l2 / n2) : 0.0;
    for (int a = 0; a < 3; ++a) t[a] *= s;
  }
}

/* Sec. 5.1, Eq. constraint_gradient: the part of a row's gradient that
   comes through the joint frame.  The frame is attached to body alpha
   (Eq. r_gradient: R_J = dR R^T with dR constant), so a row
   c = e^T R_J d = n . d (n the row's world direction, d the world gap of its
   point pair) changes by e^T dR_J d with dR_J = -R_J [omega]x, omega the
   world rotation rate of alpha's polar factor: from A = R P,
   R^T dA - dA^T R = Omega P + P Omega with Omega = R^T dR = [w]x, which is
   [(tr(P) I - P) w]x, and omega = R w.  The row gains omega . (n x d) for
   each of the nine A-entries of q_alpha (entry 3c + a: dA = e_a e_c^T). */
static void full_row_term(const double A[9], const double R[9], const double n[3],
                          const double d[3], double g[12]) {
  double P[9], Ms[9], Mi[9];
  mtm3(R, A, P);
  const double tr = P[0] + P[4] + P[8];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      Ms[3 * r + c] = (r == c ? tr : 0.0) - 0.5 * (P[3 * r + c] + P[3 * c + r]);
  inv3(Ms, Mi);
  const double m[3] = {n[1] * d[2] - n[2] * d[1], n[2] * d[0] - n[0] * d[2],
                       n[0] * d[1] - n[1] * d[0]};
  for (int c = 0; c < 3; ++c)
    for (int a = 0; a < 3; ++a) {
      double X[9] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      for (int r = 0; r < 3; ++r) X[3 * r + c] = R[3 * a + r]; /* (R^T e_a) e_c^T */
      double W[9];
      for (int r = 0; r < 3; ++r)
        for (int s = 0; s < 3; ++s) W[3 * r + s] = X[3 * r + s] - X[3 * s + r];
      const double ax[3] = {W[7], W[2], W[3]}; /* W = [ax]x */
      double w[3], om[3];
      mv3(Mi, ax, w);
      mv3(R, w, om);
      g[3 * c + a] += om[0] * m[0] + om[1] * m[1] + om[2] * m[2];
    }
}

/* ------------------------------------------------------------------ */
/* joints: Eq. ball, Eq. hinge, frozen-frame Jacobian Eq. pcpq          */
/* ------------------------------------------------------------------ */
static int is_free(const ora_scene *sc, int64_t j) { return j >= 0 && sc->fixed[j] == 0; }

static int joint_rows(const ora_scene *sc, int64_t k) {
  const int t = sc->jtype[k];
  return t == 1 || t == 3 ? 5 : (t == 2 ? 4 : 3);
}

int ora_joint_eval(const ora_scene *sc, const double *q, int64_t k, double c[5],
                   double Ga[60], double Gb[60], int32_t *rows) {
  int64_t ja = sc->body_a[k], jb = sc->body_b[k];
  int C = joint_rows(sc, k);
  if (rows) *rows = C;
  double pa[3][3], pb[3][3], dir[5][3];
  int pt[5];
  for (int i = 0; i < 3; ++i) {
    pa[0][i] = sc->anchor_a[3 * k + i];
    pb[0][i] = sc->anchor_b[3 * k + i];
  }
  const double *qa = q + 12 * ja;
  double wb1 = 1.0; /* homogeneous weight of beta's second point (0: a difference vector) */
  /* jacobian_mode 1: alpha's A and R and the world gaps of the point pairs */
  double fA[9], fR[9], fd[3][3];
  int full = 0;
  int arow3 = 1;    /* does row 3 act on alpha */
  if (sc->jtype[k] == 2) {
    /* Sec. 4.4 universal joint: R_U = [a1 x a2, a1, a2]^T with a1 fixed in
       alpha and a2 fixed in beta (Gram-Schmidt against a1, frozen at q_n);
       rows 0-2: R_U (x_alpha(p_a) - x_beta(p_b)) (a ball at the joint
       centre); row 3: a1 . (x_beta(p_b + l a2) - x_beta(p_b)), which keeps
       beta's axis in the plane normal to a1. */
    double u1[3], u2[3], A[9], R[9], Rb[9], w1[3], w2[3], r0[3], r1[3], r2[3];
    normalize3(sc->axis_a + 3 * k, u1);
    normalize3(sc->axis_b + 3 * k, u2);
    const double *qb = q + 12 * jb;
    A_of_q(qa, A);
    int st = ora_polar(A, R, NULL);
    if (st) return st;
    A_of_q(qb, A);
    st = ora_polar(A, Rb, NULL);
    if (st) return st;
    mv3(R, u1, w1);
    mv3(Rb, u2, w2);
    normalize3(w1, r1);
    double d = r1[0] * w2[0] + r1[1] * w2[1] + r1[2] * w2[2];
    double v[3] = {w2[0] - d * r1[0], w2[1] - d * r1[1], w2[2] - d * r1[2]};
    normalize3(v, r2);
    r0[0] = r1[1] * r2[2] - r1[2] * r2[1];
    r0[1] = r1[2] * r2[0] - r1[0] * r2[2];
    r0[2] = r1[0] * r2[1] - r1[1] * r2[0];
    const double l = sc->axis_len[k];
    for (int i = 0; i < 3; ++i) {
      pb[1][i] = l * u2[i];
      pa[1][i] = 0.0;
    }
    wb1 = 0.0;
    arow3 = 0;
    double d1[3], xb1[3];
    gap_of(qa, pa[0], qb, pb[0], d1);
    A_of_q(qb, A);
    mv3(A, pb[1], xb1); /* x_beta(p_b + l a2) - x_beta(p_b) = A_beta (l a2) */
    const double *rows[3] = {r0, r1, r2};
    for (int r = 0; r < 3; ++r) {
      c[r] = rows[r][0] * d1[0] + rows[r][1] * d1[1] + rows[r][2] * d1[2];
      pt[r] = 0;
      for (int a = 0; a < 3; ++a) dir[r][a] = rows[r][a];
    }
    c[3] = r1[0] * xb1[0] + r1[1] * xb1[1] + r1[2] * xb1[2];
    c[4] = 0.0;
    pt[3] = 1;
    for (int a = 0; a < 3; ++a) dir[3][a] = r1[a];
  } else if (sc->jtype[k] == 3) {
    /* Sec. 4.5 prismatic joint, frame attached to alpha (Sec. 5.1 writes a
       joint frame as a constant rotation times alpha's R^T) and frozen at
       q_n: y~ = a = R_alpha a_a (the sliding axis), x~ = R_alpha c_a made
       normal to a, z~ = x~ x y~; R_P = [x~; y~; z~] maps a to e_y.  Three
       point pairs, all on both bodies: the anchors (p_a, p_b), the on-axis
       points (p_a + l a_a, p_b + l a_b) and the off-axis points
       (p_a + l c_a, p_b + l c_b).  Rows: x~ and z~ of the anchor gap and of
       the on-axis gap (beta's axis stays on alpha's axis line), and z~ of the
       off-axis gap (no twist about a); the y~ gaps, the slide, are free. */
    double ua[3], ub[3], ca[3], cb[3], A[9], R[9], w[3], wc[3], ry[3], rx[3], rz[3];
    normalize3(sc->axis_a + 3 * k, ua);
    normalize3(sc->axis_b + 3 * k, ub);
    normalize3(sc->ref_a + 3 * k, ca);
    normalize3(sc->ref_b + 3 * k, cb);
    const double l = sc->axis_len[k];
    for (int i = 0; i < 3; ++i) {
      pa[1][i] = pa[0][i] + l * ua[i];
      pb[1][i] = pb[0][i] + l * ub[i];
      pa[2][i] = pa[0][i] + l * ca[i];
      pb[2][i] = pb[0][i] + l * cb[i];
    }
    A_of_q(qa, A);
    int st = ora_polar(A, R, NULL);
    if (st) return st;
    mv3(R, ua, w);
    normalize3(w, ry);
    mv3(R, ca, wc);
    double d = ry[0] * wc[0] + ry[1] * wc[1] + ry[2] * wc[2];
    double v[3] = {wc[0] - d * ry[0], wc[1] - d * ry[1], wc[2] - d * ry[2]};
    normalize3(v, rx);
    rz[0] = rx[1] * ry[2] - rx[2] * ry[1];
    rz[1] = rx[2] * ry[0] - rx[0] * ry[2];
    rz[2] = rx[0] * ry[1] - rx[1] * ry[0];
    const double *qb = jb == ORA_WORLD ? NULL : q + 12 * jb;
    double g[3][3];
    for (int t = 0; t < 3; ++t) gap_of(qa, pa[t], qb, pb[t], g[t]);
    const int tpt[5] = {0, 0, 1, 1, 2};
    const double *tdir[5] = {rx, rz, rx, rz, rz};
    for (int r = 0; r < 5; ++r) {
      pt[r] = tpt[r];
      c[r] = tdir[r][0] * g[pt[r]][0] + tdir[r][1] * g[pt[r]][1] + tdir[r][2] * g[pt[r]][2];
      for (int a = 0; a < 3; ++a) dir[r][a] = tdir[r][a];
    }
    if (sc->jacobian_mode == 1) {
      full = 1;
      memcpy(fA, A, sizeof(fA));
      memcpy(fR, R, sizeof(fR));
      memcpy(fd, g, sizeof(fd));
    }
  } else if (C == 3) {
    for (int r = 0; r < 3; ++r) {
      pt[r] = 0;
      for (int a = 0; a < 3; ++a) dir[r][a] = (r == a) ? 1.0 : 0.0;
    }
    gap_of(qa, pa[0], jb == ORA_WORLD ? NULL : q + 12 * jb, pb[0], c);
  } else {
    double ua[3], ub[3], A[9], R[9], a[3], ra[3], RH[9];
    normalize3(sc->axis_a + 3 * k, ua);
    normalize3(sc->axis_b + 3 * k, ub);
    double l = sc->axis_len[k];
    for (int i = 0; i < 3; ++i) {
      pa[1][i] = pa[0][i] + l * ua[i];
      pb[1][i] = pb[0][i] + l * ub[i];
    }
    /* the hinge axis is attached to body alpha (Sec. 5.1: R_H = dR_H R^alpha^T) */
    A_of_q(qa, A);
    int st = ora_polar(A, R, NULL);
    if (st) return st;
    mv3(R, ua, ra);
    normalize3(ra, a);
    if (a[1] < 0.0) { a[0] = -a[0]; a[1] = -a[1]; a[2] = -a[2]; }
    ora_hinge_frame(a, RH);
    double d1[3], d2[3], e1[3], e2[3];
    const double *qb = jb == ORA_WORLD ? NULL : q + 12 * jb;
    gap_of(qa, pa[0], qb, pb[0], d1);
    gap_of(qa, pa[1], qb, pb[1], d2);
    mv3(RH, d1, e1);
    mv3(RH, d2, e2);
    c[0] = e1[0]; c[1] = e1[1]; c[2] = e1[2];
    c[3] = e2[0]; c[4] = e2[2];
    const int rsel[5] = {0, 1, 2, 0, 2};
    for (int r = 0; r < 5; ++r) {
      pt[r] = r < 3 ? 0 : 1;
      for (int a2 = 0; a2 < 3; ++a2) dir[r][a2] = RH[3 * rsel[r] + a2];
    }
    if (sc->jacobian_mode == 1) {
      full = 1;
      memcpy(fA, A, sizeof(fA));
      memcpy(fR, R, sizeof(fR));
      memcpy(fd[0], d1, sizeof(d1));
      memcpy(fd[1], d2, sizeof(d2));
    }
  }
  if (Ga) memset(Ga, 0, 60 * sizeof(double));
  if (Gb) memset(Gb, 0, 60 * sizeof(double));
  for (int r = 0; r < C; ++r) {
    /* the universal joint's row 3 is + a1 (x) [l a2; 0] on beta, nothing on alpha */
    const int u3 = sc->jtype[k] == 2 && r == 3;
    const double sa = u3 && !arow3 ? 0.0 : 1.0, sb = u3 ? 1.0 : -1.0;
    const double wb = pt[r] == 1 ? wb1 : 1.0;
    for (int i = 0; i < 3; ++i)
      for (int a = 0; a < 3; ++a) {
        if (Ga) Ga[12 * r + 3 * i + a] = sa * pa[pt[r]][i] * dir[r][a];
        if (Gb && jb != ORA_WORLD) Gb[12 * r + 3 * i + a] = sb * pb[pt[r]][i] * dir[r][a];
      }
    for (int a = 0; a < 3; ++a) {
      if (Ga) Ga[12 * r + 9 + a] = sa * dir[r][a];
      if (Gb && jb != ORA_WORLD) Gb[12 * r + 9 + a] = sb * wb * dir[r][a];
    }
  }
  if (full && Ga)
    for (int r = 0; r < C; ++r) full_row_term(fA, fR, dir[r], fd[pt[r]], Ga + 12 * r);
  return ORA_OK;
}

int ora_joint_eval_attached(const ora_scene *sc, const double *q_ref, const double *q, int64_t k,
                            double c[5]) {
  const int t = sc->jtype[k];
  if (t == 2) return ORA_ERR_ARG;
  const int64_t ja = sc->body_a[k], jb = sc->body_b[k];
  const double *qa = q + 12 * ja, *qb = jb == ORA_WORLD ? NULL : q + 12 * jb;
  double pa[3][3], pb[3][3];
  for (int i = 0; i < 3; ++i) {
    pa[0][i] = sc->anchor_a[3 * k + i];
    pb[0][i] = sc->anchor_b[3 * k + i];
  }
  if (t == 0) {
    gap_of(qa, pa[0], qb, pb[0], c);
    return ORA_OK;
  }
  /* the frame's rows at q_ref: the translation part of alpha's Jacobian rows */
  double cr[5], Ga[60], Ar[9], Rr[9], A[9], R[9];
  int32_t C;
  int st = ora_joint_eval(sc, q_ref, k, cr, Ga, NULL, &C);
  if (st) return st;
  A_of_q(q_ref + 12 * ja, Ar);
  st = ora_polar(Ar, Rr, NULL);
  if (st) return st;
  A_of_q(qa, A);
  st = ora_polar(A, R, NULL);
  if (st) return st;
  /* the point pairs (as in ora_joint_eval) */
  double ua[3], ub[3];
  normalize3(sc->axis_a + 3 * k, ua);
  normalize3(sc->axis_b + 3 * k, ub);
  const double l = sc->axis_len[k];
  for (int i = 0; i < 3; ++i) {
    pa[1][i] = pa[0][i] + l * ua[i];
    pb[1][i] = pb[0][i] + l * ub[i];
  }
  if (t == 3) {
    double ca[3], cb[3];
    normalize3(sc->ref_a + 3 * k, ca);
    normalize3(sc->ref_b + 3 * k, cb);
    for (int i = 0; i < 3; ++i) {
      pa[2][i] = pa[0][i] + l * ca[i];
      pb[2][i] = pb[0][i] + l * cb[i];
    }
  }
  const int hpt[5] = {0, 0, 0, 1, 1}, ppt[5] = {0, 0, 1, 1, 2};
  for (int r = 0; r < C; ++r) {
    const int i = t == 3 ? ppt[r] : hpt[r];
    double n0[3] = {Ga[12 * r + 9], Ga[12 * r + 10], Ga[12 * r + 11]}, t1[3], n[3], d[3];
    mtv3(Rr, n0, t1);
    mv3(R, t1, n);
    gap_of(qa, pa[i], qb, pb[i], d);
    c[r] = n[0] * d[0] + n[1] * d[1] + n[2] * d[2];
  }
  return ORA_OK;
}

int64_t ora_dual_rows(const ora_scene *sc) {
  int64_t n = 0;
  for (int64_t k = 0; k < sc->K; ++k) n += joint_rows(sc, k);
  return n;
}

/* ------------------------------------------------------------------ */
/* topology: body -> joint incidence over free bodies                   */
/* ------------------------------------------------------------------ */
typedef struct {
  int64_t *off;   /* M+1 */
  int64_t *jnt;   /* incident joints of each free body */
  int32_t *side;  /* 0: body is alpha, 1: body is beta */
} incidence;

static int build_incidence(const ora_scene *sc, incidence *inc) {
  int64_t M = sc->M, K = sc->K;
  inc->off = (int64_t *)calloc((size_t)M + 1, sizeof(int64_t));
  for (int64_t k = 0; k < K; ++k) {
    if (is_free(sc, sc->body_a[k])) inc->off[sc->body_a[k] + 1]++;
    if (is_free(sc, sc->body_b[k])) inc->off[sc->body_b[k] + 1]++;
  }
  for (int64_t j = 0; j < M; ++j) inc->off[j + 1] += inc->off[j];
  inc->jnt = (int64_t *)malloc(sizeof(int64_t) * (size_t)(inc->off[M] + 1));
  inc->side = (int32_t *)malloc(sizeof(int32_t) * (size_t)(inc->off[M] + 1));
  int64_t *fill = (int64_t *)calloc((size_t)M, sizeof(int64_t));
  for (int64_t k = 0; k < K; ++k) {
    int64_t a = sc->body_a[k], b = sc->body_b[k];
    if (is_free(sc, a)) {
      int64_t p = inc->off[a] + fill[a]++;
      inc->jnt[p] = k;
      inc->side[p] = 0;
    }
    if (is_free(sc, b)) {
      int64_t p = inc->off[b] + fill[b]++;
      inc->jnt[p] = k;
      inc->side[p] = 1;
    }
  }
  free(fill);
  return ORA_OK;
}

static void free_incidence(incidence *inc) {
  free(inc->off);
  free(inc->jnt);
  free(inc->side);
}

static int validate(const ora_scene *sc) {
  if (sc->M < 0 || sc->K < 0 || !(sc->h > 0.0)) return ORA_ERR_ARG;
  if (sc->rotation_mode < 0 || sc->rotation_mode > 1 || sc->jacobian_mode < 0 ||
      sc->jacobian_mode > 1)
    return ORA_ERR_ARG;
  for (int64_t j = 0; j < sc->M; ++j)
    if (!(sc->mass[j] > 0.0) || !(sc->volume[j] > 0.0) || !(sc->young[j] > 0.0) ||
        !(sc->poisson[j] >= 0.0 && sc->poisson[j] < 0.5))
      return ORA_ERR_ARG;
  for (int64_t k = 0; k < sc->K; ++k) {
    int64_t a = sc->body_a[k], b = sc->body_b[k];
    if (a < 0 || a >= sc->M || b < ORA_WORLD || b >= sc->M || a == b) return ORA_ERR_ARG;
    if (sc->jtype[k] < 0 || sc->jtype[k] > 3) return ORA_ERR_ARG;
    if (!is_free(sc, a) && !is_free(sc, b)) return ORA_ERR_ARG;
    /* a universal joint's fourth row lies on body beta alone */
    if (sc->jtype[k] == 2 && !is_free(sc, b)) return ORA_ERR_ARG;
    /* the universal frame follows both bodies: no attached-frame gradient */
    if (sc->jtype[k] == 2 && sc->jacobian_mode == 1) return ORA_ERR_ARG;
  }
  return ORA_OK;
}

/* other end of joint k seen from free body j, or -1 when it is not a free body */
static int64_t other_free(const ora_scene *sc, int64_t k, int64_t j) {
  int64_t o = sc->body_a[k] == j ? sc->body_b[k] : sc->body_a[k];
  return is_free(sc, o) ? o : -1;
}

/* Chain (Sec. 5.2): free bodies form one path; joint order along it puts every
   pair of joints that share a body next to each other. order[K] on success. */
static int chain_order(const ora_scene *sc, const incidence *inc, int64_t *order) {
  int64_t M = sc->M, K = sc->K, nfree = 0, nint = 0;
  for (int64_t j = 0; j < M; ++j) nfree += is_free(sc, j);
  if (nfree == 0 || K == 0) return 0;
  for (int64_t k = 0; k < K; ++k) nint += is_free(sc, sc->body_a[k]) && is_free(sc, sc->body_b[k]);
  if (nint != nfree - 1) return 0;
  int64_t start = -1;
  for (int64_t j = 0; j < M && start < 0; ++j) {
    if (!is_free(sc, j)) continue;
    int64_t deg = 0;
    for (int64_t p = inc->off[j]; p < inc->off[j + 1]; ++p) deg += other_free(sc, inc->jnt[p], j) >= 0;
    if (deg > 2) return 0;
    if (deg <= 1) start = j;
  }
  if (start < 0) return 0;
  int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
  for (int64_t k = 0; k < K; ++k) pos[k] = -1;
  int64_t n = 0, cur = start, prev_joint = -1, visited = 0;
  while (cur >= 0) {
    visited++;
    /* world/fixed joints of this body first, then the joint to the next body */
    for (int64_t p = inc->off[cur]; p < inc->off[cur + 1]; ++p) {
      int64_t k = inc->jnt[p];
      if (other_free(sc, k, cur) < 0 && pos[k] < 0) { pos[k] = n; order[n++] = k; }
    }
    int64_t next = -1, nj = -1;
    for (int64_t p = inc->off[cur]; p < inc->off[cur + 1]; ++p) {
      int64_t k = inc->jnt[p];
      if (k != prev_joint && other_free(sc, k, cur) >= 0 && pos[k] < 0) { next = other_free(sc, k, cur); nj = k; }
    }
    if (nj >= 0) { pos[nj] = n; order[n++] = nj; }
    prev_joint = nj;
    cur = next;
  }
  int ok = (visited == nfree) && (n == K);
  /* block tridiagonal iff the joints of each body sit at adjacent positions */
  for (int64_t j = 0; ok && j < M; ++j) {
    if (!is_free(sc, j)) continue;
    int64_t cnt = inc->off[j + 1] - inc->off[j];
    if (cnt > 2) ok = 0;
    if (cnt == 2) {
      int64_t d = pos[inc->jnt[inc->off[j]]] - pos[inc->jnt[inc->off[j] + 1]];
      if (d != 1 && d != -1) ok = 0;
    }
  }
  free(pos);
  return ok;
}

/* Tree / forest (Sec. 5.3): internal joints form a forest; joints to the world
   or to fixed bodies only at one body per component, which becomes its root.
   Outputs BFS order, parent body and parent joint per free body. */
static int tree_order(const ora_scene *sc, const incidence *inc, int64_t *bfs, int64_t *parent,
                      int64_t *pjoint, int64_t *nbfs) {
  int64_t M = sc->M;
  int64_t *comp_root = (int64_t *)malloc(sizeof(int64_t) * (size_t)M);
  for (int64_t j = 0; j < M; ++j) { parent[j] = -2; pjoint[j] = -1; comp_root[j] = -1; }
  int ok = 1;
  int64_t n = 0;
  /* component discovery by BFS from each unvisited free body */
  int64_t *seen = (int64_t *)calloc((size_t)M, sizeof(int64_t));
  for (int64_t s = 0; s < M && ok; ++s) {
    if (!is_free(sc, s) || seen[s]) continue;
    /* collect component */
    int64_t c0 = n, tail = n;
    bfs[tail++] = s;
    seen[s] = 1;
    int64_t head = c0, root = -1, nroot_cand = 0, edges2 = 0;
    while (head < tail) {
      int64_t j = bfs[head++];
      int has_world = 0;
      for (int64_t p = inc->off[j]; p < inc->off[j + 1]; ++p) {
        int64_t k = inc->jnt[p], o = other_free(sc, k, j);
        if (o < 0) { has_world = 1; continue; }
        edges2++;
        if (!seen[o]) { seen[o] = 1; bfs[tail++] = o; }
      }
      if (has_world) { nroot_cand++; root = j; }
    }
    int64_t ncomp = tail - c0;
    if (edges2 / 2 != ncomp - 1 || nroot_cand > 1) { ok = 0; break; }
    if (root < 0) root = s;
    /* BFS from the root to set parents */
    for (int64_t i = c0; i < tail; ++i) seen[bfs[i]] = 2;
    int64_t h2 = c0, t2 = c0;
    bfs[t2++] = root;
    seen[root] = 3;
    parent[root] = -1;
    while (h2 < t2) {
      int64_t j = bfs[h2++];
      for (int64_t p = inc->off[j]; p < inc->off[j + 1]; ++p) {
        int64_t k = inc->jnt[p], o = other_free(sc, k, j);
        if (o < 0 || seen[o] == 3) continue;
        seen[o] = 3;
        parent[o] = j;
        pjoint[o] = k;
        bfs[t2++] = o;
      }
    }
    n = t2;
  }
  *nbfs = n;
  free(seen);
  free(comp_root);
  return ok;
}

int ora_topology(const ora_scene *sc) {
  if (validate(sc)) return -ORA_ERR_ARG;
  incidence inc;
  build_incidence(sc, &inc);
  int64_t *o = (int64_t *)malloc(sizeof(int64_t) * (size_t)(sc->K + 1));
  int64_t *b = (int64_t *)malloc(sizeof(int64_t) * (size_t)(sc->M + 1));
  int64_t *p = (int64_t *)malloc(sizeof(int64_t) * (size_t)(sc->M + 1));
  int64_t *pj = (int64_t *)malloc(sizeof(int64_t) * (size_t)(sc->M + 1));
  int64_t nb;
  int t = 3;
  if (chain_order(sc, &inc, o)) t = 1;
  else if (tree_order(sc, &inc, b, p, pj, &nb)) t = 2;
  free(o); free(b); free(p); free(pj);
  free_incidence(&inc);
  return t;
}

/* ------------------------------------------------------------------ */
/* per-body operators                                                  */
/* ------------------------------------------------------------------ */
typedef struct {
  double *L;   /* 144 per body: Cholesky of Hbar_A */
  double *R;   /* 9 per body */
  double *f;   /* 12 per body (world) */
  double *u;   /* 12 per body: unconstrained solve H_A^{-1} f */
} body_data;

/* diag4(R) applies R to each of the four 3-blocks of a 12-vector */
static void diag4(const double R[9], const double *x, double *y) {
  for (int b = 0; b < 4; ++b) mv3(R, x + 3 * b, y + 3 * b);
}
static void diag4T(const double R[9], const double *x, double *y) {
  for (int b = 0; b < 4; ++b) mtv3(R, x + 3 * b, y + 3 * b);
}

/* H_A^{-1} x = diag4(R) Hbar^{-1} diag4(R^T) x  (Eq. abd_final) */
static void hinv_apply(const double *L, const double R[9], const double *x, double *y) {
  double t[12], s[12];
  diag4T(R, x, t);
  chol_solve(12, L, t, s);
  diag4(R, s, y);
}

/* H_A x = diag4(R) L L^T diag4(R^T) x */
static void h_apply(const double *L, const double R[9], const double *x, double *y) {
  double t[12], s[12];
  diag4T(R, x, t);
  for (int r = 0; r < 12; ++r) {
    double v = 0.0;
    for (int k = r; k < 12; ++k) v += L[12 * k + r] * t[k];
    s[r] = v;
  }
  for (int r = 0; r < 12; ++r) {
    double v = 0.0;
    for (int k = 0; k <= r; ++k) v += L[12 * r + k] * s[k];
    t[r] = v;
  }
  diag4(R, t, y);
}

/* W = L^{-1} diag4(R^T) g for one constraint row g (12) */
static void w_row(const double *L, const double R[9], const double *g, double *w) {
  double t[12];
  diag4T(R, g, t);
  lower_solve(12, L, t, w);
}

/* ------------------------------------------------------------------ */
/* dual matrix in block-sparse form (Eq. dual, Fig. dual_mat)           */
/* ------------------------------------------------------------------ */
typedef struct {
  int64_t *off;   /* K+1 */
  int64_t *col;   /* neighbour joints, sorted */
  int64_t *boff;  /* offset of each block in val */
  double *val;
} bsr;

static int cmp_i64(const void *a, const void *b) {
  int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
  return (x > y) - (x < y);
}

static void bsr_build(const ora_scene *sc, const incidence *inc, bsr *S) {
  int64_t K = sc->K;
  int64_t *cnt = (int64_t *)calloc((size_t)K + 1, sizeof(int64_t));
  for (int64_t k = 0; k < K; ++k) {
    int64_t ends[2] = {sc->body_a[k], sc->body_b[k]};
    for (int e = 0; e < 2; ++e)
      if (is_free(sc, ends[e])) cnt[k + 1] += inc->off[ends[e] + 1] - inc->off[ends[e]];
  }
  for (int64_t k = 0; k < K; ++k) cnt[k + 1] += cnt[k];
  int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(cnt[K] + 1));
  S->off = (int64_t *)calloc((size_t)K + 1, sizeof(int64_t));
  for (int64_t k = 0; k < K; ++k) {
    int64_t n = 0, base = cnt[k];
    int64_t ends[2] = {sc->body_a[k], sc->body_b[k]};
    for (int e = 0; e < 2; ++e)
      if (is_free(sc, ends[e]))
        for (int64_t p = inc->off[ends[e]]; p < inc->off[ends[e] + 1]; ++p) tmp[base + n++] = inc->jnt[p];
    qsort(tmp + base, (size_t)n, sizeof(int64_t), cmp_i64);
    int64_t u = 0;
    for (int64_t i = 0; i < n; ++i)
      if (i == 0 || tmp[base + i] != tmp[base + i - 1]) tmp[base + u++] = tmp[base + i];
    S->off[k + 1] = u;
  }
  for (int64_t k = 0; k < K; ++k) S->off[k + 1] += S->off[k];
  S->col = (int64_t *)malloc(sizeof(int64_t) * (size_t)(S->off[K] + 1));
  S->boff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(S->off[K] + 1));
  int64_t vo = 0;
  for (int64_t k = 0; k < K; ++k) {
    int64_t n = S->off[k + 1] - S->off[k];
    for (int64_t i = 0; i < n; ++i) {
      int64_t kk = tmp[cnt[k] + i];
      S->col[S->off[k] + i] = kk;
      S->boff[S->off[k] + i] = vo;
      vo += (int64_t)joint_rows(sc, k) * joint_rows(sc, kk);
    }
  }
  S->val = (double *)calloc((size_t)vo + 1, sizeof(double));
  free(tmp);
  free(cnt);
}

static double *bsr_block(const bsr *S, int64_t k, int64_t kk) {
  int64_t lo = S->off[k], hi = S->off[k + 1] - 1;
  while (lo <= hi) {
    int64_t mid = (lo + hi) / 2;
    if (S->col[mid] == kk) return S->val + S->boff[mid];
    if (S->col[mid] < kk) lo = mid + 1;
    else hi = mid - 1;
  }
  return NULL;
}

static void bsr_free(bsr *S) {
  free(S->off); free(S->col); free(S->boff); free(S->val);
}

/* ------------------------------------------------------------------ */
/* the step                                                            */
/* ------------------------------------------------------------------ */
typedef struct {
  int64_t *roff;  /* K+1 row offsets */
  double *c;      /* rows: constraint values C(q_n) */
  double *b;      /* rows: dual rhs G u + c */
  double *Ga, *Gb; /* 60 per joint */
} joint_data;

static double *G_of(const joint_data *jd, int64_t k, int side) {
  return (side == 0 ? jd->Ga : jd->Gb) + 60 * k;
}

/* S_{k k'} += sum over free bodies j shared by k and k' of W_kj^T W_k'j  (Eq. dual) */
static int assemble_S(const ora_scene *sc, const incidence *inc, const body_data *bd,
                      const joint_data *jd, bsr *S, double *Sd, int64_t nrows) {
  double *W = (double *)malloc(sizeof(double) * 12 * 5 * 64);
  for (int64_t j = 0; j < sc->M; ++j) {
    if (!is_free(sc, j)) continue;
    int64_t n = inc->off[j + 1] - inc->off[j];
    if (n > 64) { free(W); return ORA_ERR_ARG; }
    for (int64_t p = 0; p < n; ++p) {
      int64_t k = inc->jnt[inc->off[j] + p];
      int C = joint_rows(sc, k);
      const double *G = G_of(jd, k, inc->side[inc->off[j] + p]);
      for (int r = 0; r < C; ++r) w_row(bd->L + 144 * j, bd->R + 9 * j, G + 12 * r, W + 60 * p + 12 * r);
    }
    for (int64_t p = 0; p < n; ++p) {
      int64_t k = inc->jnt[inc->off[j] + p];
      int C = joint_rows(sc, k);
      for (int64_t pp = 0; pp < n; ++pp) {
        int64_t kk = inc->jnt[inc->off[j] + pp];
        int CC = joint_rows(sc, kk);
        double *blk = S ? bsr_block(S, k, kk) : NULL;
        for (int r = 0; r < C; ++r)
          for (int s = 0; s < CC; ++s) {
            double v = 0.0;
            for (int i = 0; i < 12; ++i) v += W[60 * p + 12 * r + i] * W[60 * pp + 12 * s + i];
            if (blk) blk[r * CC + s] += v;
            if (Sd) Sd[(jd->roff[k] + r) * nrows + jd->roff[kk] + s] += v;
          }
      }
    }
  }
  free(W);
  return ORA_OK;
}

/* Block Thomas on the block-tridiagonal dual (Eq. chain-btd) */
static int solve_chain(const ora_scene *sc, const bsr *S, const joint_data *jd,
                       const int64_t *order, double *lambda) {
  int64_t K = sc->K;
  double *Dp = (double *)malloc(sizeof(double) * 25 * (size_t)K);  /* Cholesky of D'_i */
  double *bp = (double *)malloc(sizeof(double) * 5 * (size_t)K);
  double Dm[25], Y[25], tmp[5];
  int st = ORA_OK;
  for (int64_t i = 0; i < K && !st; ++i) {
    int64_t k = order[i];
    int C = joint_rows(sc, k);
    memcpy(Dm, bsr_block(S, k, k), sizeof(double) * C * C);
    for (int r = 0; r < C; ++r) bp[5 * i + r] = jd->b[jd->roff[k] + r];
    if (i > 0) {
      /* D'_i = D_i - B_{i-1}^T D'_{i-1}^{-1} B_{i-1};  b'_i = b_i - B_{i-1}^T D'_{i-1}^{-1} b'_{i-1} */
      int64_t kp = order[i - 1];
      int Cp = joint_rows(sc, kp);
      const double *B = bsr_block(S, kp, k); /* Cp x C */
      for (int s = 0; s < C; ++s) {
        double col[5];
        for (int r = 0; r < Cp; ++r) col[r] = B[r * C + s];
        chol_solve(Cp, Dp + 25 * (i - 1), col, Y + 5 * s); /* Y[:,s] = D'^{-1} B[:,s] */
      }
      for (int r = 0; r < C; ++r)
        for (int s = 0; s < C; ++s) {
          double v = 0.0;
          for (int t = 0; t < Cp; ++t) v += B[t * C + r] * Y[5 * s + t];
          Dm[r * C + s] -= v;
        }
      chol_solve(Cp, Dp + 25 * (i - 1), bp + 5 * (i - 1), tmp);
      for (int r = 0; r < C; ++r) {
        double v = 0.0;
        for (int t = 0; t < Cp; ++t) v += B[t * C + r] * tmp[t];
        bp[5 * i + r] -= v;
      }
    }
    st = cholesky(C, Dm, Dp + 25 * i);
  }
  if (!st) {
    for (int64_t i = K - 1; i >= 0; --i) {
      int64_t k = order[i];
      int C = joint_rows(sc, k);
      double rhs[5];
      for (int r = 0; r < C; ++r) rhs[r] = bp[5 * i + r];
      if (i < K - 1) {
        int64_t kn = order[i + 1];
        int Cn = joint_rows(sc, kn);
        const double *B = bsr_block(S, k, kn); /* C x Cn */
        for (int r = 0; r < C; ++r)
          for (int s = 0; s < Cn; ++s) rhs[r] -= B[r * Cn + s] * lambda[jd->roff[kn] + s];
      }
      chol_solve(C, Dp + 25 * i, rhs, lambda + jd->roff[k]);
    }
  }
  free(Dp);
  free(bp);
  return st;
}

/* block-Jacobi preconditioned CG on the dual matrix (graph case) */
static void bsr_mv(const ora_scene *sc, const bsr *S, const joint_data *jd, const double *x, double *y) {
  for (int64_t k = 0; k < sc->K; ++k) {
    int C = joint_rows(sc, k);
    for (int r = 0; r < C; ++r) y[jd->roff[k] + r] = 0.0;
    for (int64_t p = S->off[k]; p < S->off[k + 1]; ++p) {
      int64_t kk = S->col[p];
      int CC = joint_rows(sc, kk);
      const double *B = S->val + S->boff[p];
      for (int r = 0; r < C; ++r) {
        double v = 0.0;
        for (int s = 0; s < CC; ++s) v += B[r * CC + s] * x[jd->roff[kk] + s];
        y[jd->roff[k] + r] += v;
      }
    }
  }
}

static int solve_cg(const ora_scene *sc, const bsr *S, const joint_data *jd, int64_t n,
                    double *x, ora_stats *st) {
  int64_t K = sc->K;
  double *Lp = (double *)malloc(sizeof(double) * 25 * (size_t)K);
  for (int64_t k = 0; k < K; ++k) {
    int C = joint_rows(sc, k);
    if (cholesky(C, bsr_block(S, k, k), Lp + 25 * k)) { free(Lp); return ORA_ERR_NOT_SPD; }
  }
  double *r = (double *)malloc(sizeof(double) * n), *z = (double *)malloc(sizeof(double) * n);
  double *p = (double *)malloc(sizeof(double) * n), *Ap = (double *)malloc(sizeof(double) * n);
  double bn = 0.0;
  for (int64_t i = 0; i < n; ++i) { x[i] = 0.0; bn += jd->b[i] * jd->b[i]; }
  bn = sqrt(bn);
  int64_t it = 0, maxit = 20 * n + 1000;
  double rel = 0.0;
  for (int restart = 0; restart < 4; ++restart) {
    bsr_mv(sc, S, jd, x, Ap);
    double rn = 0.0;
    for (int64_t i = 0; i < n; ++i) { r[i] = jd->b[i] - Ap[i]; rn += r[i] * r[i]; }
    rel = bn > 0 ? sqrt(rn) / bn : 0.0;
    if (rel <= 1e-14) break;
    for (int64_t k = 0; k < K; ++k) chol_solve(joint_rows(sc, k), Lp + 25 * k, r + jd->roff[k], z + jd->roff[k]);
    double rz = 0.0;
    for (int64_t i = 0; i < n; ++i) { p[i] = z[i]; rz += r[i] * z[i]; }
    for (; it < maxit; ++it) {
      bsr_mv(sc, S, jd, p, Ap);
      double pAp = 0.0;
      for (int64_t i = 0; i < n; ++i) pAp += p[i] * Ap[i];
      double alpha = rz / pAp;
      rn = 0.0;
      for (int64_t i = 0; i < n; ++i) {
        x[i] += alpha * p[i];
        r[i] -= alpha * Ap[i];
        rn += r[i] * r[i];
      }
      if (bn == 0.0 || sqrt(rn) <= 1e-14 * bn) { ++it; break; }
      for (int64_t k = 0; k < K; ++k) chol_solve(joint_rows(sc, k), Lp + 25 * k, r + jd->roff[k], z + jd->roff[k]);
      double rz2 = 0.0;
      for (int64_t i = 0; i < n; ++i) rz2 += r[i] * z[i];
      double beta = rz2 / rz;
      rz = rz2;
      for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    /* true residual of the iterate */
    bsr_mv(sc, S, jd, x, Ap);
    rn = 0.0;
    for (int64_t i = 0; i < n; ++i) { double t = jd->b[i] - Ap[i]; rn += t * t; }
    rel = bn > 0 ? sqrt(rn) / bn : 0.0;
    if (rel <= 1e-14 || it >= maxit) break;
  }
  if (st) { st->cg_iters = (int32_t)it; st->cg_rel_residual = rel; }
  free(r); free(z); free(p); free(Ap); free(Lp);
  return ORA_OK;
}

/* Sec. 5.3, exact body-space reading of Alg. 2 / Eq. module3-kkt:
   upward   Hhat_p += P_j^T D_j^{-1} P_j,  fhat_p -= P_j^T D_j^{-1} (G_j Hhat_j^{-1} fhat_j + c_j),
            D_j = G_j Hhat_j^{-1} G_j^T, G_j = dC_j/dq_j, P_j = dC_j/dq_p;
   downward lambda_j = D_j^{-1}(G_j Hhat_j^{-1} fhat_j + c_j + P_j dq_p),
            dq_j = Hhat_j^{-1}(fhat_j - G_j^T lambda_j). */
static int solve_tree(const ora_scene *sc, const incidence *inc, const body_data *bd,
                      const joint_data *jd, double *lambda) {
  int64_t M = sc->M;
  int64_t *bfs = (int64_t *)malloc(sizeof(int64_t) * (size_t)(M + 1));
  int64_t *par = (int64_t *)malloc(sizeof(int64_t) * (size_t)(M + 1));
  int64_t *pj = (int64_t *)malloc(sizeof(int64_t) * (size_t)(M + 1));
  int64_t nb = 0;
  if (!tree_order(sc, inc, bfs, par, pj, &nb)) {
    free(bfs); free(par); free(pj);
    return ORA_ERR_TOPOLOGY;
  }
  double *Hh = (double *)malloc(sizeof(double) * 144 * (size_t)M);
  double *fh = (double *)malloc(sizeof(double) * 12 * (size_t)M);
  double *Lh = (double *)malloc(sizeof(double) * 144 * (size_t)M);
  double *y = (double *)malloc(sizeof(double) * 12 * (size_t)M);
  /* rows eliminated at a body: its parent joint, or the world joints of a root */
  int64_t nmax = 5;
  for (int64_t i = 0; i < nb; ++i) {
    int64_t j = bfs[i], n = 0;
    if (par[j] >= 0) continue;
    for (int64_t q2 = inc->off[j]; q2 < inc->off[j + 1]; ++q2)
      if (other_free(sc, inc->jnt[q2], j) < 0) n += joint_rows(sc, inc->jnt[q2]);
    if (n > nmax) nmax = n;
  }
  if (nmax > 64) { free(bfs); free(par); free(pj); return ORA_ERR_ARG; }
  double *X = (double *)malloc(sizeof(double) * 12 * nmax * (size_t)M); /* Hhat^{-1} G^T */
  double *LD = (double *)malloc(sizeof(double) * nmax * nmax * (size_t)M);
  double *e = (double *)malloc(sizeof(double) * nmax * (size_t)M);
  double *dq = (double *)malloc(sizeof(double) * 12 * (size_t)M);
  int st = ORA_OK;
  /* Hhat_j = H_j (world frame, dense), fhat_j = f_j */
  for (int64_t i = 0; i < nb; ++i) {
    int64_t j = bfs[i];
    double Hb[144], T[144], Hw[144];
    const double *R = bd->R + 9 * j;
    ora_system_matrix(sc->mass[j], sc->second_moment + 6 * j, sc->volume[j], sc->young[j],
                      sc->poisson[j], sc->h, Hb);
    /* Hw = diag4(R) Hb diag4(R^T) */
    for (int c = 0; c < 12; ++c) {
      double col[12], rc[12];
      for (int r = 0; r < 12; ++r) col[r] = Hb[12 * r + c];
      diag4(R, col, rc);
      for (int r = 0; r < 12; ++r) T[12 * r + c] = rc[r];
    }
    for (int r = 0; r < 12; ++r) {
      double row[12], rr[12];
      for (int c = 0; c < 12; ++c) row[c] = T[12 * r + c];
      diag4(R, row, rr);
      for (int c = 0; c < 12; ++c) Hw[12 * r + c] = rr[c];
    }
    memcpy(Hh + 144 * j, Hw, sizeof(Hw));
    memcpy(fh + 12 * j, bd->f + 12 * j, 12 * sizeof(double));
  }
  /* rows attached to body j that go up (its parent joint) or to the world (root) */
  for (int64_t ii = nb - 1; ii >= 0 && !st; --ii) {
    int64_t j = bfs[ii];
    /* gather the constraint rows eliminated at j */
    double Gj[64 * 12], Pj[64 * 12], cj[64];
    int n = 0;
    int64_t p = par[j];
    if (p >= 0) {
      int64_t k = pj[j];
      int side = sc->body_a[k] == j ? 0 : 1;
      int C = joint_rows(sc, k);
      for (int r = 0; r < C; ++r) {
        memcpy(Gj + 12 * (n + r), G_of(jd, k, side) + 12 * r, 12 * sizeof(double));
        memcpy(Pj + 12 * (n + r), G_of(jd, k, 1 - side) + 12 * r, 12 * sizeof(double));
        cj[n + r] = sc->residual_rhs ? jd->c[jd->roff[k] + r] : 0.0;
      }
      n += C;
    } else {
      for (int64_t q2 = inc->off[j]; q2 < inc->off[j + 1]; ++q2) {
        int64_t k = inc->jnt[q2];
        if (other_free(sc, k, j) >= 0) continue;
        int C = joint_rows(sc, k);
        if (n + C > 64) { st = ORA_ERR_ARG; break; }
        for (int r = 0; r < C; ++r) {
          memcpy(Gj + 12 * (n + r), G_of(jd, k, inc->side[q2]) + 12 * r, 12 * sizeof(double));
          memset(Pj + 12 * (n + r), 0, 12 * sizeof(double));
          cj[n + r] = sc->residual_rhs ? jd->c[jd->roff[k] + r] : 0.0;
        }
        n += C;
      }
    }
    if (st) break;
    double *L = Lh + 144 * j;
    st = cholesky(12, Hh + 144 * j, L);
    if (st) break;
    chol_solve(12, L, fh + 12 * j, y + 12 * j);
    double *Xj = X + 12 * nmax * j;
    for (int r = 0; r < n; ++r) chol_solve(12, L, Gj + 12 * r, Xj + 12 * r); /* row r of X^T */
    double D[64 * 64];
    for (int r = 0; r < n; ++r)
      for (int s = 0; s < n; ++s) {
        double v = 0.0;
        for (int i = 0; i < 12; ++i) v += Gj[12 * r + i] * Xj[12 * s + i];
        D[r * n + s] = v;
      }
    double *ej = e + nmax * j;
    for (int r = 0; r < n; ++r) {
      double v = cj[r];
      for (int i = 0; i < 12; ++i) v += Gj[12 * r + i] * y[12 * j + i];
      ej[r] = v;
    }
    if (n > 0) {
      double Ld[64 * 64];
      st = cholesky(n, D, Ld);
      if (st) break;
      memcpy(LD + nmax * nmax * j, Ld, sizeof(double) * n * n);
    }
    if (p >= 0) {
      /* Hhat_p += P^T D^{-1} P ; fhat_p -= P^T D^{-1} e */
      double DinvP[64 * 12], col[64], sol[64], Dinve[64];
      for (int i = 0; i < 12; ++i) {
        for (int r = 0; r < n; ++r) col[r] = Pj[12 * r + i];
        chol_solve(n, LD + nmax * nmax * j, col, sol);
        for (int r = 0; r < n; ++r) DinvP[12 * r + i] = sol[r];
      }
      chol_solve(n, LD + nmax * nmax * j, ej, Dinve);
      for (int a = 0; a < 12; ++a) {
        for (int b = 0; b < 12; ++b) {
          double v = 0.0;
          for (int r = 0; r < n; ++r) v += Pj[12 * r + a] * DinvP[12 * r + b];
          Hh[144 * p + 12 * a + b] += v;
        }
        double v = 0.0;
        for (int r = 0; r < n; ++r) v += Pj[12 * r + a] * Dinve[r];
        fh[12 * p + a] -= v;
      }
    }
  }
  /* downward pass */
  for (int64_t ii = 0; ii < nb && !st; ++ii) {
    int64_t j = bfs[ii];
    int64_t p = par[j];
    double rhs[64], lam[64];
    int n = 0;
    if (p >= 0) {
      int64_t k = pj[j];
      int side = sc->body_a[k] == j ? 0 : 1;
      int C = joint_rows(sc, k);
      const double *P = G_of(jd, k, 1 - side);
      for (int r = 0; r < C; ++r) {
        double v = e[nmax * j + r];
        for (int i = 0; i < 12; ++i) v += P[12 * r + i] * dq[12 * p + i];
        rhs[r] = v;
      }
      n = C;
      chol_solve(n, LD + nmax * nmax * j, rhs, lam);
      for (int r = 0; r < C; ++r) lambda[jd->roff[k] + r] = lam[r];
    } else {
      for (int64_t q2 = inc->off[j]; q2 < inc->off[j + 1]; ++q2) {
        int64_t k = inc->jnt[q2];
        if (other_free(sc, k, j) >= 0) continue;
        n += joint_rows(sc, k);
      }
      if (n > 0) {
        chol_solve(n, LD + nmax * nmax * j, e + nmax * j, lam);
        int m = 0;
        for (int64_t q2 = inc->off[j]; q2 < inc->off[j + 1]; ++q2) {
          int64_t k = inc->jnt[q2];
          if (other_free(sc, k, j) >= 0) continue;
          int C = joint_rows(sc, k);
          for (int r = 0; r < C; ++r) lambda[jd->roff[k] + r] = lam[m + r];
          m += C;
        }
      }
    }
    for (int i = 0; i < 12; ++i) {
      double v = y[12 * j + i];
      for (int r = 0; r < n; ++r) v -= X[12 * nmax * j + 12 * r + i] * lam[r];
      dq[12 * j + i] = v;
    }
  }
  free(bfs); free(par); free(pj); free(Hh); free(fh); free(Lh); free(y);
  free(X); free(LD); free(e); free(dq);
  return st;
}

static int setup(const ora_scene *sc, const double *q, const double *qd, body_data *bd,
                 joint_data *jd) {
  int64_t M = sc->M, K = sc->K;
  bd->L = (double *)calloc(144 * (size_t)M + 1, sizeof(double));
  bd->R = (double *)calloc(9 * (size_t)M + 1, sizeof(double));
  bd->f = (double *)calloc(12 * (size_t)M + 1, sizeof(double));
  bd->u = (double *)calloc(12 * (size_t)M + 1, sizeof(double));
  jd->roff = (int64_t *)calloc((size_t)K + 1, sizeof(int64_t));
  for (int64_t k = 0; k < K; ++k) jd->roff[k + 1] = jd->roff[k] + joint_rows(sc, k);
  int64_t n = jd->roff[K];
  jd->c = (double *)calloc((size_t)n + 1, sizeof(double));
  jd->b = (double *)calloc((size_t)n + 1, sizeof(double));
  jd->Ga = (double *)calloc(60 * (size_t)K + 1, sizeof(double));
  jd->Gb = (double *)calloc(60 * (size_t)K + 1, sizeof(double));
  for (int64_t j = 0; j < 12 * M; ++j)
    if (!isfinite(q[j]) || !isfinite(qd[j])) return ORA_ERR_NONFINITE;
  for (int64_t j = 0; j < M; ++j) {
    if (!is_free(sc, j)) continue;
    double H[144];
    ora_system_matrix(sc->mass[j], sc->second_moment + 6 * j, sc->volume[j], sc->young[j],
                      sc->poisson[j], sc->h, H);
    int st = cholesky(12, H, bd->L + 144 * j);
    if (st) return st;
    st = ora_body_rhs(sc, j, q, qd, bd->f + 12 * j, bd->R + 9 * j);
    if (st) return st;
    if (sc->rotation_mode == 1) {
      /* u by Alg. 1; f becomes H_A u, so that the dual rhs, the tree
         elimination and the recovery of dq, which reach u through the
         linear H_A, all use Alg. 1's u */
      double A[9];
      A_of_q(q + 12 * j, A);
      ora_alg1_solve(bd->L + 144 * j, A, bd->f + 12 * j, bd->u + 12 * j);
      h_apply(bd->L + 144 * j, bd->R + 9 * j, bd->u + 12 * j, bd->f + 12 * j);
    } else {
      hinv_apply(bd->L + 144 * j, bd->R + 9 * j, bd->f + 12 * j, bd->u + 12 * j);
    }
  }
  for (int64_t k = 0; k < K; ++k) {
    double c[5];
    int32_t C;
    int st = ora_joint_eval(sc, q, k, c, jd->Ga + 60 * k, jd->Gb + 60 * k, &C);
    if (st) return st;
    int64_t a = sc->body_a[k], b = sc->body_b[k];
    for (int r = 0; r < C; ++r) {
      double v = sc->residual_rhs ? c[r] : 0.0;
      if (is_free(sc, a))
        for (int i = 0; i < 12; ++i) v += jd->Ga[60 * k + 12 * r + i] * bd->u[12 * a + i];
      if (is_free(sc, b))
        for (int i = 0; i < 12; ++i) v += jd->Gb[60 * k + 12 * r + i] * bd->u[12 * b + i];
      jd->c[jd->roff[k] + r] = c[r];
      jd->b[jd->roff[k] + r] = v;
    }
  }
  return ORA_OK;
}

static void teardown(body_data *bd, joint_data *jd) {
  free(bd->L); free(bd->R); free(bd->f); free(bd->u);
  free(jd->roff); free(jd->c); free(jd->b); free(jd->Ga); free(jd->Gb);
}

int ora_assemble_dense(const ora_scene *sc, const double *q, const double *qd, double *Hw,
                       double *f, double *G, double *c) {
  int st = validate(sc);
  if (st) return st;
  body_data bd;
  joint_data jd;
  st = setup(sc, q, qd, &bd, &jd);
  if (!st) {
    int64_t M = sc->M, n = jd.roff[sc->K];
    for (int64_t j = 0; j < M; ++j) {
      double *H = Hw + 144 * j;
      memset(H, 0, 144 * sizeof(double));
      memset(f + 12 * j, 0, 12 * sizeof(double));
      if (!is_free(sc, j)) continue;
      /* H_A = diag4(R) L L^T diag4(R^T), built column by column via H e_c */
      for (int cidx = 0; cidx < 12; ++cidx) {
        double ecol[12] = {0}, t[12], s[12], y[12];
        ecol[cidx] = 1.0;
        diag4T(bd.R + 9 * j, ecol, t);
        const double *L = bd.L + 144 * j;
        for (int r = 0; r < 12; ++r) { /* s = L^T t */
          double v = 0.0;
          for (int k = r; k < 12; ++k) v += L[12 * k + r] * t[k];
          s[r] = v;
        }
        for (int r = 0; r < 12; ++r) { /* t = L s */
          double v = 0.0;
          for (int k = 0; k <= r; ++k) v += L[12 * r + k] * s[k];
          t[r] = v;
        }
        diag4(bd.R + 9 * j, t, y);
        for (int r = 0; r < 12; ++r) H[12 * r + cidx] = y[r];
      }
      memcpy(f + 12 * j, bd.f + 12 * j, 12 * sizeof(double));
    }
    memset(G, 0, sizeof(double) * (size_t)n * 12 * (size_t)M);
    for (int64_t k = 0; k < sc->K; ++k) {
      int C = joint_rows(sc, k);
      int64_t a = sc->body_a[k], b = sc->body_b[k];
      for (int r = 0; r < C; ++r) {
        int64_t row = jd.roff[k] + r;
        c[row] = jd.c[row];
        if (is_free(sc, a))
          for (int i = 0; i < 12; ++i) G[row * 12 * M + 12 * a + i] = jd.Ga[60 * k + 12 * r + i];
        if (is_free(sc, b))
          for (int i = 0; i < 12; ++i) G[row * 12 * M + 12 * b + i] = jd.Gb[60 * k + 12 * r + i];
      }
    }
  }
  teardown(&bd, &jd);
  return st;
}

int ora_step(const ora_scene *sc, int32_t solver, const double *q, const double *qd,
             double *q_out, double *qd_out, double *lambda, ora_stats *stats) {
  int st = validate(sc);
  if (st) return st;
  int64_t M = sc->M, K = sc->K;
  body_data bd;
  joint_data jd;
  incidence inc;
  ora_stats local;
  memset(&local, 0, sizeof(local));
  st = setup(sc, q, qd, &bd, &jd);
  build_incidence(sc, &inc);
  int64_t n = jd.roff[K];
  double *lam = (double *)calloc((size_t)n + 1, sizeof(double));
  int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(K + 1));
  int is_chain = (!st && K > 0) ? chain_order(sc, &inc, order) : 0;
  if (!st && K > 0) {
    int use = solver;
    if (use == ORA_SOLVER_AUTO) {
      if (is_chain) use = ORA_SOLVER_CHAIN;
      else {
        int64_t *b1 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(M + 1));
        int64_t *b2 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(M + 1));
        int64_t *b3 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(M + 1));
        int64_t nb;
        use = tree_order(sc, &inc, b1, b2, b3, &nb) ? ORA_SOLVER_TREE : ORA_SOLVER_CG;
        free(b1); free(b2); free(b3);
      }
    }
    local.solver_used = use;
    if (use == ORA_SOLVER_TREE) {
      st = solve_tree(sc, &inc, &bd, &jd, lam);
    } else if (use == ORA_SOLVER_DENSE) {
      if (n > 6000) st = ORA_ERR_ARG;
      else {
        double *Sd = (double *)calloc((size_t)(n * n), sizeof(double));
        double *Ld = (double *)malloc(sizeof(double) * (size_t)(n * n));
        st = assemble_S(sc, &inc, &bd, &jd, NULL, Sd, n);
        if (!st) st = cholesky((int)n, Sd, Ld);
        if (!st) chol_solve((int)n, Ld, jd.b, lam);
        free(Sd);
        free(Ld);
      }
    } else {
      bsr S;
      bsr_build(sc, &inc, &S);
      st = assemble_S(sc, &inc, &bd, &jd, &S, NULL, n);
      if (!st) {
        if (use == ORA_SOLVER_CHAIN) st = is_chain ? solve_chain(sc, &S, &jd, order, lam) : ORA_ERR_TOPOLOGY;
        else st = solve_cg(sc, &S, &jd, n, lam, &local);
      }
      bsr_free(&S);
    }
  }
  if (!st) {
    /* Eq. recover-dq-explicit: dq_j = H_j^{-1}(f_j - sum_k G_kj^T lambda_k), then
       implicit Euler q_{n+1} = q_n + dq, qdot_{n+1} = dq / h */
    double *dq = (double *)calloc(12 * (size_t)M + 1, sizeof(double));
    for (int64_t j = 0; j < M; ++j) {
      if (!is_free(sc, j)) continue;
      double g[12] = {0}, w[12];
      for (int64_t p = inc.off[j]; p < inc.off[j + 1]; ++p) {
        int64_t k = inc.jnt[p];
        const double *G = G_of(&jd, k, inc.side[p]);
        int C = joint_rows(sc, k);
        for (int r = 0; r < C; ++r)
          for (int i = 0; i < 12; ++i) g[i] += G[12 * r + i] * lam[jd.roff[k] + r];
      }
      double fg[12];
      for (int i = 0; i < 12; ++i) fg[i] = bd.f[12 * j + i] - g[i];
      hinv_apply(bd.L + 144 * j, bd.R + 9 * j, fg, w);
      for (int i = 0; i < 12; ++i) dq[12 * j + i] = w[i];
    }
    for (int64_t j = 0; j < M; ++j)
      for (int i = 0; i < 12; ++i) {
        if (is_free(sc, j)) {
          q_out[12 * j + i] = q[12 * j + i] + dq[12 * j + i];
          qd_out[12 * j + i] = dq[12 * j + i] / sc->h;
        } else {
          q_out[12 * j + i] = q[12 * j + i];
          qd_out[12 * j + i] = qd[12 * j + i];
        }
      }
    /* residuals (Table 1 |r|): linearized |G dq + c| and nonlinear |C(q_{n+1})| */
    double lin = 0.0, nl = 0.0;
    for (int64_t k = 0; k < K && !st; ++k) {
      int C = joint_rows(sc, k);
      int64_t a = sc->body_a[k], b = sc->body_b[k];
      for (int r = 0; r < C; ++r) {
        double v = jd.c[jd.roff[k] + r];
        if (is_free(sc, a))
          for (int i = 0; i < 12; ++i) v += jd.Ga[60 * k + 12 * r + i] * dq[12 * a + i];
        if (is_free(sc, b))
          for (int i = 0; i < 12; ++i) v += jd.Gb[60 * k + 12 * r + i] * dq[12 * b + i];
        if (fabs(v) > lin) lin = fabs(v);
      }
      double c2[5];
      int32_t C2;
      st = ora_joint_eval(sc, q_out, k, c2, NULL, NULL, &C2);
      for (int r = 0; r < C2 && !st; ++r)
        if (fabs(c2[r]) > nl) nl = fabs(c2[r]);
    }
    local.lin_residual = lin;
    local.joint_residual = nl;
    if (lambda) memcpy(lambda, lam, sizeof(double) * (size_t)n);
    free(dq);
  }
  if (stats) *stats = local;
  free(lam);
  free(order);
  free_incidence(&inc);
  teardown(&bd, &jd);
  return st;
}
