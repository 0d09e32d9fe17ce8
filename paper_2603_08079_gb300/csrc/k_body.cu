// Per-body and per-joint kernels of one M-ABD step (FP64):
//   k_body_prep  (Sec. 3.3-3.4)  R = polar(A), rest-frame rhs, ubar = Hbar^{-1} fbar
//   k_joint_prep (Sec. 4.2-4.3, Sec. 5.1 Eq. pcpq)  C(q_n), hinge frame, dual rhs
//   k_backprop   (Sec. 5.2 Eq. recover-dq-explicit) dq, q, qdot
//   k_residuals  (Table 1 |r|)  max |G dq + C(q_n)| and max |C(q_{n+1})|
// Variants: Alg. 1 for the unconstrained solve (StepParams::rot_norm) and the
// frame term of the full constraint gradient (DevJoints::qf non-null).
#include "mabd_device.cuh"

namespace mabd {

// Alg. 1 (Sec. 3.4, Eq. len_preserving): the unconstrained solve with each
// 3-block taken to the rest frame as A^T f_k rescaled to |f_k| and back as
// A dp_k rescaled to |dp_k| (a zero block stays zero).  fb is the rest-frame
// force of the polar form, so R fb_k is the world block f_k; ub receives the
// rest-frame copy R^T u_k of the result, as the rest of the step expects.
__device__ __forceinline__ void alg1_solve(const double A[9], const double R[9], const double fb[12],
                                           const double h[16], double ub[12]) {
  double ft[12], dp[12];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double f[3], t[3];
    mv3(R, fb + 3 * k, f);
    mtv3(A, f, t);
    const double l2 = f[0] * f[0] + f[1] * f[1] + f[2] * f[2];
    const double n2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    const double sc = n2 > 0.0 ? sqrt(l2 / n2) : 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) ft[3 * k + a] = sc * t[a];
  }
  hinv_apply(h, ft, dp);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double w[3];
    mv3(A, dp + 3 * k, w);
    const double l2 = dp[3 * k] * dp[3 * k] + dp[3 * k + 1] * dp[3 * k + 1] + dp[3 * k + 2] * dp[3 * k + 2];
    const double n2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    const double sc = n2 > 0.0 ? sqrt(l2 / n2) : 0.0;
    w[0] *= sc; w[1] *= sc; w[2] *= sc;
    mtv3(R, w, ub + 3 * k);
  }
}

// One thread per body.  f = M_A qdot/h + [0; m g] - diag4(R)[V vec(P(R^T A)); 0]
// (Eq. newton_abd rhs at x = x_n, co-rotated linear elasticity of Sec. 3.3),
// expressed in the rest frame: fbar = diag4(R^T)(M_A qdot/h + [0; m g]) - [V vec P; 0];
// ubar = Hbar^{-1} fbar (Eq. abd_final).
// NORM: Alg. 1 for the unconstrained solve (its own instantiation: the
// default keeps its register count)
template <bool NORM>
__global__ void __launch_bounds__(128) k_body_prep(DevBodies B, StepParams p, int *status,
                                                      unsigned long long *iters) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= B.M) return;
  const int M = B.M;
  double q[12], qd[12], A[9], R[9];
  load12(B.q, M, j, q);
  A_from_q(q, A);
  int nit = 0;
  int st = polar3(A, R, &nit);
  if (iters) count_add(iters, (unsigned)nit);
  if (st) {
    set_status(status, st);
#pragma unroll
    for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0) ? 1.0 : 0.0;
  }
  if (B.fixed[j]) {  // no unknowns; its rotation may still orient a hinge
#pragma unroll
    for (int i = 0; i < 9; ++i) B.R[(size_t)i * M + j] = R[i];
#pragma unroll
    for (int i = 0; i < 12; ++i) B.ubar[(size_t)i * M + j] = 0.0;
    return;
  }
  load12(B.qd, M, j, qd);
  const double s0 = ldg(B.sig + j), s1 = ldg(B.sig + M + j), s2 = ldg(B.sig + 2 * (size_t)M + j);
  const double m = ldg(B.mass + j);
  const double sh0 = s0 * p.inv_h, sh1 = s1 * p.inv_h, sh2 = s2 * p.inv_h, mh = m * p.inv_h;
  const double vmu = ldg(B.vmu + j), vlam = ldg(B.vlam + j);
  // world-frame inertial + gravity force, then rotate each 3-block by R^T
  double fw[12];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    fw[a] = sh0 * qd[a];
    fw[3 + a] = sh1 * qd[3 + a];
    fw[6 + a] = sh2 * qd[6 + a];
    fw[9 + a] = mh * qd[9 + a] + m * p.g[a];
  }
  double fb[12];
#pragma unroll
  for (int blk = 0; blk < 4; ++blk) mtv3(R, fw + 3 * blk, fb + 3 * blk);
  // F = R^T A ; V P(F) = vmu (F + F^T - 2I) + vlam tr(F - I) I ; fbar_el = -vec(V P)
  double F[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) F[3 * r + c] = R[r] * A[c] + R[3 + r] * A[3 + c] + R[6 + r] * A[6 + c];
  const double tr = vlam * (F[0] + F[4] + F[8] - 3.0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      // vec(P)[3i+a] = P(a,i)
      double P = vmu * (F[3 * a + i] + F[3 * i + a] - (a == i ? 2.0 : 0.0)) + (a == i ? tr : 0.0);
      fb[3 * i + a] -= P;
    }
  double h[16], u[12];
  load_hinv(B, j, h);
  if (NORM) alg1_solve(A, R, fb, h, u);
  else hinv_apply(h, fb, u);
#pragma unroll
  for (int i = 0; i < 9; ++i) B.R[(size_t)i * M + j] = R[i];
#pragma unroll
  for (int i = 0; i < 12; ++i) B.ubar[(size_t)i * M + j] = u[i];
}

// displacement of rest point p of body j under the unconstrained solve:
// J(p) u = R (J(p) ubar) with u = diag4(R) ubar
__device__ __forceinline__ void u_at(const double R[9], const double ub[12], const double p[3],
                                     double x[3]) {
  double l[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) l[a] = ub[a] * p[0] + ub[3 + a] * p[1] + ub[6 + a] * p[2] + ub[9 + a];
  mv3(R, l, x);
}

// MABD_JACOBIAN_FULL: the frame term of each of a hinge's or prismatic
// joint's five rows on body a (frame rows RJ[3 * sel[r] ..], world gaps
// dv[r]).  Stores qh_r = K R_a^T (n_r x d_r) (zero when a is not free) and
// returns in ext[r] the term's share of the dual rhs, qh_r . axial(U - U^T)
// with U the 3x3 block of a's unconstrained rest-frame solve ua.
__device__ __forceinline__ void full_rows(const double qa[12], const double Ra[9], const double ua[12],
                                          const double RJ[9], const double *const dv[5], uint8_t fl,
                                          double *qf, int K, int k, const int sel[5], double ext[5]) {
  double KRt[9] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, w[3] = {0.0, 0.0, 0.0};
  const bool af = (fl & JF_A_FREE) != 0;
  if (af) {
    double A[9];
    A_from_q(qa, A);
    full_frame_map(A, Ra, KRt);
    skew_axial(ua, w);
  }
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const double n[3] = {RJ[3 * sel[r]], RJ[3 * sel[r] + 1], RJ[3 * sel[r] + 2]};
    double qh[3];
    full_row_vec(KRt, n, dv[r], qh);
#pragma unroll
    for (int i = 0; i < 3; ++i) qf[(size_t)(3 * r + i) * K + k] = qh[i];
    ext[r] = af ? qh[0] * w[0] + qh[1] * w[1] + qh[2] * w[2] : 0.0;
  }
}

// One thread per joint: C(q_n) (Eq. ball / hinge / universal / prismatic),
// the joint frame taken from the bodies' rotations (hinge: axis sign chosen
// so that a_y >= 0), and the dual rhs b = G u + C(q_n) with G the
// frozen-frame Jacobian (Eq. pcpq).
template <bool XJ>
__global__ void __launch_bounds__(128) k_joint_prep(DevBodies B, DevJoints J, StepParams p,
                                                    int *status) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= J.K) return;
  const int k = ordered(J.order, t);
  const int K = J.K, M = B.M;
  const int type = J.type[k];
  const int ia = J.ja[k], ib = J.jb[k];
  const uint8_t fl = J.flags[k];
  if (!MABD_INDEX_OK(ia, M, status) || ((fl & JF_B_BODY) && !MABD_INDEX_OK(ib, M, status))) return;
  double qa[12], pa1[3], pb1[3];
  load12(B.q, M, ia, qa);
  load3(J.pa1, K, k, pa1);
  load3(J.pb1, K, k, pb1);
  double qb[12];
  if (fl & JF_B_BODY) load12(B.q, M, ib, qb);
  double Ra[9], ua[12], Rb[9], ub[12];
  load_R(B.R, M, ia, Ra);
  if (fl & JF_A_FREE) load12(B.ubar, M, ia, ua);
  if (fl & JF_B_FREE) {
    load_R(B.R, M, ib, Rb);
    load12(B.ubar, M, ib, ub);
  }
  double d1[3];
  gap_of(qa, pa1, (fl & JF_B_BODY) ? qb : nullptr, pb1, d1);
  // displacement difference of the first points under u
  double g1[3] = {0.0, 0.0, 0.0};
  {
    double t[3];
    if (fl & JF_A_FREE) {
      u_at(Ra, ua, pa1, t);
      g1[0] += t[0]; g1[1] += t[1]; g1[2] += t[2];
    }
    if (fl & JF_B_FREE) {
      u_at(Rb, ub, pb1, t);
      g1[0] -= t[0]; g1[1] -= t[1]; g1[2] -= t[2];
    }
  }
  const double rr = p.residual_rhs ? 1.0 : 0.0;
  if (type == 0) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      J.c[(size_t)r * K + k] = d1[r];
      J.b[(size_t)r * K + k] = g1[r] + rr * d1[r];
    }
    return;
  }
  if ((XJ && type == 2)) {
    // universal (Sec. 4.4): ball rows in R_U, row 3 = a1 . A_b (l a2) on b alone
    double uax[3], vb[3], RU[9], Rbb[9], Ab[9], xb[3], lb[3], gb3[3];
    load3(J.ua, K, k, uax);
    load3(J.pb2, K, k, vb);
    if (fl & JF_B_FREE) {
#pragma unroll
      for (int i = 0; i < 9; ++i) Rbb[i] = Rb[i];
    } else {
      load_R(B.R, M, ib, Rbb);
    }
    universal_frame(Ra, uax, Rbb, vb, RU);
    A_from_q(qb, Ab);
    mv3(Ab, vb, xb);
    double c1[3], e1[3];
    mv3(RU, d1, c1);
    mv3(RU, g1, e1);
    // b's displacement of its axis vector under u: R_b (J_0(l a2) ubar_b)
    gb3[0] = gb3[1] = gb3[2] = 0.0;
    if (fl & JF_B_FREE) {
#pragma unroll
      for (int a2 = 0; a2 < 3; ++a2) lb[a2] = ub[a2] * vb[0] + ub[3 + a2] * vb[1] + ub[6 + a2] * vb[2];
      mv3(Rb, lb, gb3);
    }
    const double c3 = RU[3] * xb[0] + RU[4] * xb[1] + RU[5] * xb[2];
    const double e3 = RU[3] * gb3[0] + RU[4] * gb3[1] + RU[5] * gb3[2];
    const double cc[4] = {c1[0], c1[1], c1[2], c3};
    const double gg[4] = {e1[0], e1[1], e1[2], e3};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      J.c[(size_t)r * K + k] = cc[r];
      J.b[(size_t)r * K + k] = gg[r] + rr * cc[r];
    }
    J.c[(size_t)4 * K + k] = 0.0;
    J.b[(size_t)4 * K + k] = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) J.RH[(size_t)i * K + k] = RU[i];
    return;
  }
  if ((XJ && type == 3)) {
    // prismatic (Sec. 4.5): x~ and z~ rows of the anchor and on-axis gaps,
    // the z~ row of the off-axis gap, in R_P attached to a
    double uax[3], P[2][3], Q[2][3], ca[3], RP[9], dd[2][3], gg[2][3];
    load3(J.ua, K, k, uax);
    load3(J.pa2, K, k, P[0]);
    load3(J.pb2, K, k, Q[0]);
    load3(J.pa3, K, k, P[1]);
    load3(J.pb3, K, k, Q[1]);
#pragma unroll
    for (int a = 0; a < 3; ++a) ca[a] = P[1][a] - pa1[a];
    prismatic_frame(Ra, uax, ca, RP);
#pragma unroll
    for (int t2 = 0; t2 < 2; ++t2) {
      gap_of(qa, P[t2], (fl & JF_B_BODY) ? qb : nullptr, Q[t2], dd[t2]);
      gg[t2][0] = gg[t2][1] = gg[t2][2] = 0.0;
      double t[3];
      if (fl & JF_A_FREE) {
        u_at(Ra, ua, P[t2], t);
        gg[t2][0] += t[0]; gg[t2][1] += t[1]; gg[t2][2] += t[2];
      }
      if (fl & JF_B_FREE) {
        u_at(Rb, ub, Q[t2], t);
        gg[t2][0] -= t[0]; gg[t2][1] -= t[1]; gg[t2][2] -= t[2];
      }
    }
    const double *x = RP, *z = RP + 6;
    const double *dv[5] = {d1, d1, dd[0], dd[0], dd[1]};
    const double *gv[5] = {g1, g1, gg[0], gg[0], gg[1]};
    double ext[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (J.qf) {
      const int sel[5] = {0, 2, 0, 2, 2};
      full_rows(qa, Ra, ua, RP, dv, fl, J.qf, K, k, sel, ext);
    }
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      const double *e = (r == 0 || r == 2) ? x : z;
      const double c = e[0] * dv[r][0] + e[1] * dv[r][1] + e[2] * dv[r][2];
      const double g = e[0] * gv[r][0] + e[1] * gv[r][1] + e[2] * gv[r][2];
      J.c[(size_t)r * K + k] = c;
      J.b[(size_t)r * K + k] = (g + ext[r]) + rr * c;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) J.RH[(size_t)i * K + k] = RP[i];
    return;
  }
  // hinge
  double pa2[3], pb2[3], uax[3], a[3], RH[9];
  load3(J.pa2, K, k, pa2);
  load3(J.pb2, K, k, pb2);
  load3(J.ua, K, k, uax);
  mv3(Ra, uax, a);
  {
    double n = rsqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    double sgn = a[1] < 0.0 ? -n : n;
    a[0] *= sgn; a[1] *= sgn; a[2] *= sgn;
  }
  hinge_frame(a, RH);
  double d2[3];
  gap_of(qa, pa2, (fl & JF_B_BODY) ? qb : nullptr, pb2, d2);
  double g2[3] = {0.0, 0.0, 0.0};
  {
    double t[3];
    if (fl & JF_A_FREE) {
      u_at(Ra, ua, pa2, t);
      g2[0] += t[0]; g2[1] += t[1]; g2[2] += t[2];
    }
    if (fl & JF_B_FREE) {
      u_at(Rb, ub, pb2, t);
      g2[0] -= t[0]; g2[1] -= t[1]; g2[2] -= t[2];
    }
  }
  double c1[3], e1[3], c2[3], e2[3];
  mv3(RH, d1, c1);
  mv3(RH, g1, e1);
  mv3(RH, d2, c2);
  mv3(RH, g2, e2);
  const double cc[5] = {c1[0], c1[1], c1[2], c2[0], c2[2]};
  const double gg[5] = {e1[0], e1[1], e1[2], e2[0], e2[2]};
  double ext[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (J.qf) {
    const double *dv[5] = {d1, d1, d1, d2, d2};
    const int sel[5] = {0, 1, 2, 0, 2};
    full_rows(qa, Ra, ua, RH, dv, fl, J.qf, K, k, sel, ext);
  }
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    J.c[(size_t)r * K + k] = cc[r];
    J.b[(size_t)r * K + k] = (gg[r] + ext[r]) + rr * cc[r];
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) J.RH[(size_t)i * K + k] = RH[i];
}

// One thread per body: g = diag4(R^T) sum_k G_kj^T lambda_k accumulated point by
// point (a row with point p and world direction d contributes [p;1] (x) R^T d),
// dq = diag4(R)(ubar - Hbar^{-1} g) (Eq. recover-dq-explicit), then the
// implicit Euler update q += dq, qdot = dq / h.
template <bool XJ>
__global__ void __launch_bounds__(128) k_backprop(DevBodies B, DevJoints J, DevIncidence I,
                                                  StepParams p) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B.M) return;
  const int j = ordered(B.order, t);
  if (B.fixed[j]) return;
  const int M = B.M, K = J.K;
  double R[9], g[12];
  load_R(B.R, M, j, R);
#pragma unroll
  for (int i = 0; i < 12; ++i) g[i] = 0.0;
  const int e0 = I.off[j], e1 = I.off[j + 1];
  for (int e = e0; e < e1; ++e) {
    const int k = I.joint[e];
    const int side = I.side[e];
    const int type = J.type[k];
    const double sgn = side == 0 ? 1.0 : -1.0;
    double lam[5];
#pragma unroll
    for (int r = 0; r < 5; ++r) lam[r] = J.lambda[(size_t)r * K + k];
    double F1[3], F2[3] = {0.0, 0.0, 0.0}, F3[3] = {0.0, 0.0, 0.0};
    double P1[3], P2[3], P3[3];
    if (side == 0) {
      load3(J.pa1, K, k, P1);
    } else {
      load3(J.pb1, K, k, P1);
    }
    double w2 = 1.0;  // translation weight of the second point (universal: 0)
    if (type == 0) {
      F1[0] = lam[0]; F1[1] = lam[1]; F1[2] = lam[2];
    } else {
      double RH[9];
      load_R(J.RH, K, k, RH);
      double l3[3] = {lam[0], lam[1], lam[2]};
      mtv3(RH, l3, F1);
      if (type == 1) {
#pragma unroll
        for (int a = 0; a < 3; ++a) F2[a] = lam[3] * RH[a] + lam[4] * RH[6 + a];
      } else if ((XJ && type == 3)) {
        // prismatic: x~, z~ at the anchors, x~, z~ on the axis, z~ off it
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          F1[a] = lam[0] * RH[a] + lam[1] * RH[6 + a];
          F2[a] = lam[2] * RH[a] + lam[3] * RH[6 + a];
          F3[a] = lam[4] * RH[6 + a];
        }
        if (side == 0) load3(J.pa3, K, k, P3);
        else load3(J.pb3, K, k, P3);
      } else if (XJ && side == 1) {
        // universal row 3 on b: + a1 lambda_3 at the point difference l a2
#pragma unroll
        for (int a = 0; a < 3; ++a) F2[a] = -lam[3] * RH[3 + a];  // sgn = -1 on b cancels below
        w2 = 0.0;
      }
      if (side == 0) load3(J.pa2, K, k, P2);
      else load3(J.pb2, K, k, P2);
    }
    double f1[3];
    mtv3(R, F1, f1);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double v = sgn * f1[a];
      g[a] += P1[0] * v;
      g[3 + a] += P1[1] * v;
      g[6 + a] += P1[2] * v;
      g[9 + a] += v;
    }
    if (type == 1 || (XJ && type == 3) || ((XJ && type == 2) && side == 1)) {
      double f2[3];
      mtv3(R, F2, f2);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double v = sgn * f2[a];
        g[a] += P2[0] * v;
        g[3 + a] += P2[1] * v;
        g[6 + a] += P2[2] * v;
        g[9 + a] += w2 * v;
      }
    }
    if (J.qf && side == 0 && (type == 1 || (XJ && type == 3))) {
      // MABD_JACOBIAN_FULL: the rows' frame term on body a
#pragma unroll
      for (int r = 0; r < 5; ++r) {
        double qh[3];
        load_qf(J.qf, K, k, r, qh);
        add_skew_force(qh, lam[r], g);
      }
    }
    if ((XJ && type == 3)) {
      double f3[3];
      mtv3(R, F3, f3);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double v = sgn * f3[a];
        g[a] += P3[0] * v;
        g[3 + a] += P3[1] * v;
        g[6 + a] += P3[2] * v;
        g[9 + a] += v;
      }
    }
  }
  double h[16], w[12], ub[12];
  load_hinv(B, j, h);
  hinv_apply(h, g, w);
  load12(B.ubar, M, j, ub);
#pragma unroll
  for (int i = 0; i < 12; ++i) ub[i] -= w[i];
#pragma unroll
  for (int blk = 0; blk < 4; ++blk) {
    double dq[3];
    mv3(R, ub + 3 * blk, dq);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const size_t o = (size_t)(3 * blk + a) * M + j;
      B.q[o] += dq[a];
      B.qd[o] = dq[a] * p.inv_h;
    }
  }
}

// One thread per joint (statistics only): linearized residual G dq + C(q_n)
// with dq = h qdot_{n+1}, and the nonlinear residual C(q_{n+1}) with the hinge
// frame re-evaluated from body a's new rotation.
template <bool XJ>
__device__ __forceinline__ void joint_residuals(const DevBodies &B, const DevJoints &J,
                                                const StepParams &p, int k, int *status,
                                                double &lin_out, double &nl_out) {
  const int K = J.K, M = B.M;
  const int type = J.type[k];
  const int ia = J.ja[k], ib = J.jb[k];
  const uint8_t fl = J.flags[k];
  const int C = joint_nrows(type);
  const int npt = type == 0 ? 1 : ((XJ && type == 3) ? 3 : 2);
  double qa[12], qb[12], dqa[12], dqb[12];
  load12(B.q, M, ia, qa);
  load12(B.qd, M, ia, dqa);
  if (fl & JF_B_BODY) {
    load12(B.q, M, ib, qb);
    load12(B.qd, M, ib, dqb);
  }
  double P[3][3], Q[3][3];
  load3(J.pa1, K, k, P[0]);
  load3(J.pb1, K, k, Q[0]);
  if (type != 0) {
    load3(J.pa2, K, k, P[1]);
    load3(J.pb2, K, k, Q[1]);
  }
  if ((XJ && type == 3)) {
    load3(J.pa3, K, k, P[2]);
    load3(J.pb3, K, k, Q[2]);
  }
  double RH[9];
  if (type != 0) load_R(J.RH, K, k, RH);
  // linearized residual with the frozen frame of this step
  double lin = 0.0;
  double da[3][3], db[3][3];
  for (int pt = 0; pt < npt; ++pt) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      da[pt][a] = 0.0;
      db[pt][a] = 0.0;
    }
    if (fl & JF_A_FREE) {
#pragma unroll
      for (int a = 0; a < 3; ++a)
        da[pt][a] = p.h * (dqa[a] * P[pt][0] + dqa[3 + a] * P[pt][1] + dqa[6 + a] * P[pt][2] + dqa[9 + a]);
    }
    if (fl & JF_B_FREE) {
      // (the universal joint's second point on b is a difference: no translation)
      const double wt = ((XJ && type == 2) && pt == 1) ? 0.0 : 1.0;
#pragma unroll
      for (int a = 0; a < 3; ++a)
        db[pt][a] = p.h * (dqb[a] * Q[pt][0] + dqb[3 + a] * Q[pt][1] + dqb[6 + a] * Q[pt][2] + wt * dqb[9 + a]);
    }
  }
  // MABD_JACOBIAN_FULL: axial(X - X^T) of a's rest-frame displacement block
  double wa[3] = {0.0, 0.0, 0.0};
  const bool full = J.qf && (fl & JF_A_FREE) && (type == 1 || (XJ && type == 3));
  if (full) {
    double Ra[9], xr[12];
    load_R(B.R, M, ia, Ra);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double dA[3] = {p.h * dqa[3 * c], p.h * dqa[3 * c + 1], p.h * dqa[3 * c + 2]};
      mtv3(Ra, dA, xr + 3 * c);
    }
    xr[9] = xr[10] = xr[11] = 0.0;
    skew_axial(xr, wa);
  }
  for (int r = 0; r < C; ++r) {
    double d[3];
    row_dir(type, RH, r, d);
    const int pt = (XJ && type == 3) ? (r >> 1) : (r < 3 ? 0 : 1);
    double v = J.c[(size_t)r * K + k];
    if (full) {
      double qh[3];
      load_qf(J.qf, K, k, r, qh);
      v += qh[0] * wa[0] + qh[1] * wa[1] + qh[2] * wa[2];
    }
    if ((XJ && type == 2) && r == 3) {
#pragma unroll
      for (int a = 0; a < 3; ++a) v += d[a] * db[1][a];
    } else {
#pragma unroll
      for (int a = 0; a < 3; ++a) v += d[a] * (da[pt][a] - db[pt][a]);
    }
    lin = fmax(lin, fabs(v));
  }
  // nonlinear residual at q_{n+1}
  double nl = 0.0;
  double d1[3], d2[3];
  const double *qbp = (fl & JF_B_BODY) ? qb : nullptr;
  gap_of(qa, P[0], qbp, Q[0], d1);
  if (type == 0) {
    nl = fmax(fabs(d1[0]), fmax(fabs(d1[1]), fabs(d1[2])));
  } else if ((XJ && type == 2)) {
    double A[9], Ra[9], Rb[9], u[3], RU[9], xb[3], c1[3];
    A_from_q(qa, A);
    int st = polar3(A, Ra);
    if (st) set_status(status, st);
    A_from_q(qb, A);
    st = polar3(A, Rb);
    if (st) set_status(status, st);
    load3(J.ua, K, k, u);
    universal_frame(Ra, u, Rb, Q[1], RU);
    mv3(RU, d1, c1);
    mv3(A, Q[1], xb);
    const double c3 = RU[3] * xb[0] + RU[4] * xb[1] + RU[5] * xb[2];
    nl = fmax(fmax(fabs(c1[0]), fabs(c1[1])), fmax(fabs(c1[2]), fabs(c3)));
  } else if ((XJ && type == 3)) {
    double A[9], Ra[9], u[3], ca[3], RP[9], d3[3];
    A_from_q(qa, A);
    int st = polar3(A, Ra);
    if (st) set_status(status, st);
    load3(J.ua, K, k, u);
#pragma unroll
    for (int a = 0; a < 3; ++a) ca[a] = P[2][a] - P[0][a];
    prismatic_frame(Ra, u, ca, RP);
    gap_of(qa, P[1], qbp, Q[1], d2);
    gap_of(qa, P[2], qbp, Q[2], d3);
    const double *x = RP, *z = RP + 6;
    const double *dv[5] = {d1, d1, d2, d2, d3};
    for (int r = 0; r < 5; ++r) {
      const double *e = (r == 0 || r == 2) ? x : z;
      nl = fmax(nl, fabs(e[0] * dv[r][0] + e[1] * dv[r][1] + e[2] * dv[r][2]));
    }
  } else {
    double A[9], R[9], u[3], a[3], RH1[9];
    A_from_q(qa, A);
    int st = polar3(A, R);
    if (st) set_status(status, st);
    load3(J.ua, K, k, u);
    mv3(R, u, a);
    double n = rsqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    double sgn = a[1] < 0.0 ? -n : n;
    a[0] *= sgn; a[1] *= sgn; a[2] *= sgn;
    hinge_frame(a, RH1);
    gap_of(qa, P[1], qbp, Q[1], d2);
    double c1[3], c2[3];
    mv3(RH1, d1, c1);
    mv3(RH1, d2, c2);
    nl = fmax(fmax(fabs(c1[0]), fabs(c1[1])), fmax(fabs(c1[2]), fmax(fabs(c2[0]), fabs(c2[2]))));
  }
  lin_out = lin;
  nl_out = nl;
}

template <bool XJ>
__global__ void __launch_bounds__(128) k_residuals(DevBodies B, DevJoints J, StepParams p,
                                                   unsigned long long *maxbits, int *status) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double lin = 0.0, nl = 0.0;
  if (t < J.K) joint_residuals<XJ>(B, J, p, ordered(J.order, t), status, lin, nl);
  // warp-level max first (all lanes take part), then one atomic per warp
  for (int o = 16; o > 0; o >>= 1) {
    lin = fmax(lin, __shfl_xor_sync(0xffffffffu, lin, o));
    nl = fmax(nl, __shfl_xor_sync(0xffffffffu, nl, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(maxbits, lin);
    atomic_max_nonneg(maxbits + 1, nl);
  }
}

// ---------------------------------------------------------------------------
// state transfer between the caller's layout and the device layout
// ---------------------------------------------------------------------------
// stage: the caller's arrays as given, q then qdot, each [M][12] in user body
// order; the device keeps [12][M] in internal order (boi: internal -> user)
__global__ void k_state_check(const double *stage, size_t n, int *flag) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    if (!isfinite(stage[i])) atomicOr(flag, 1);
}

// bodies kept in their principal frame (non-diagonal second moment given):
// A_lib = A_caller V on the way in, A_caller = A_lib V^T on the way out, for
// q and qdot alike (V row-major, 9 per body in user order)
__global__ void __launch_bounds__(128) k_stage_frames(double *stage, int M, const double *frames,
                                                      const uint8_t *has_frame, int to_lib) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M || !has_frame[j]) return;
  double V[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) V[i] = frames[(size_t)9 * j + i];
  for (int part = 0; part < 2; ++part) {
    double *x = stage + (size_t)part * 12 * M + (size_t)12 * j;
    double t[9];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int r = 0; r < 3; ++r)
        t[3 * c + r] = to_lib ? x[r] * V[c] + x[3 + r] * V[3 + c] + x[6 + r] * V[6 + c]
                              : x[r] * V[3 * c] + x[3 + r] * V[3 * c + 1] + x[6 + r] * V[3 * c + 2];
#pragma unroll
    for (int i = 0; i < 9; ++i) x[i] = t[i];
  }
}

__global__ void __launch_bounds__(128) k_state_in(const double *stage, const int32_t *boi, DevBodies B) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int M = B.M;
  if (i >= M) return;
  const size_t u = (size_t)boi[i];
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    B.q[(size_t)c * M + i] = stage[12 * u + c];
    B.qd[(size_t)c * M + i] = stage[12 * (size_t)M + 12 * u + c];
  }
}

__global__ void __launch_bounds__(128) k_state_out(DevBodies B, const int32_t *boi, double *stage) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int M = B.M;
  if (i >= M) return;
  const size_t u = (size_t)boi[i];
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    stage[12 * u + c] = B.q[(size_t)c * M + i];
    stage[12 * (size_t)M + 12 * u + c] = B.qd[(size_t)c * M + i];
  }
}

static inline int nblk(int n, int t) { return (n + t - 1) / t; }

void launch_state_check(const double *stage, size_t n, int *flag, cudaStream_t s) {
  if (n) k_state_check<<<1216, 256, 0, s>>>(stage, n, flag);
}

void launch_state_in(const double *stage, const int32_t *boi, const DevBodies &B, cudaStream_t s) {
  if (B.M > 0) k_state_in<<<nblk(B.M, 128), 128, 0, s>>>(stage, boi, B);
}

void launch_state_out(const DevBodies &B, const int32_t *boi, double *stage, cudaStream_t s) {
  if (B.M > 0) k_state_out<<<nblk(B.M, 128), 128, 0, s>>>(B, boi, stage);
}

void launch_stage_frames(double *stage, int M, const double *frames, const uint8_t *has_frame,
                         bool to_lib, cudaStream_t s) {
  if (M > 0) k_stage_frames<<<nblk(M, 128), 128, 0, s>>>(stage, M, frames, has_frame, to_lib ? 1 : 0);
}

void launch_body_prep(const DevBodies &B, const StepParams &p, int *status, cudaStream_t s,
                      unsigned long long *iters) {
  if (B.M <= 0) return;
  if (p.rot_norm) k_body_prep<true><<<nblk(B.M, 128), 128, 0, s>>>(B, p, status, iters);
  else k_body_prep<false><<<nblk(B.M, 128), 128, 0, s>>>(B, p, status, iters);
}

void launch_joint_prep(const DevBodies &B, const DevJoints &J, const StepParams &p, int *status,
                       cudaStream_t s) {
  if (J.K == 0) return;
  if (J.xj) k_joint_prep<true><<<nblk(J.K, 128), 128, 0, s>>>(B, J, p, status);
  else k_joint_prep<false><<<nblk(J.K, 128), 128, 0, s>>>(B, J, p, status);
}

void launch_backprop(const DevBodies &B, const DevJoints &J, const DevIncidence &I,
                     const StepParams &p, int * /*status*/, cudaStream_t s) {
  if (B.M == 0) return;
  if (J.xj) k_backprop<true><<<nblk(B.M, 128), 128, 0, s>>>(B, J, I, p);
  else k_backprop<false><<<nblk(B.M, 128), 128, 0, s>>>(B, J, I, p);
}

void launch_residuals(const DevBodies &B, const DevJoints &J, const StepParams &p,
                      unsigned long long *maxbits, int *status, cudaStream_t s) {
  if (J.K == 0) return;
  if (J.xj) k_residuals<true><<<nblk(J.K, 128), 128, 0, s>>>(B, J, p, maxbits, status);
  else k_residuals<false><<<nblk(J.K, 128), 128, 0, s>>>(B, J, p, maxbits, status);
}

}  // namespace mabd
