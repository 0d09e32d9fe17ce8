// Mixed-precision forms of the step (chains, trees and the PCG path share
// these kernels).  The step solves the same linearized KKT system as the FP64
// form (Eq. newton_abd with the frozen-frame Jacobian of Eq. pcpq):
//     H dq + G^T lambda = f,     G dq = -C(q_n)
// by iterative refinement:
//   approximate solve  u = H^{-1} f, Gram blocks, then back-propagation
//                      dq = u - H^{-1} G^T lambda (Sec. 5.2), with every
//                      per-body and per-joint product in FP32, and the dual
//                      solve by the chain's block cyclic reduction (FP64, or
//                      FP32 in MABD_MIXED_FP32_DUAL), the tree's FP32
//                      elimination, or FP32 PCG on graphs;
//   correction sweep   FP64 residuals r_p = f - H dq - G^T lambda and
//                      r_d = -C - G dq, then the same approximate solve for
//                      (r_p, r_d) (through the stored factors on chains).
// Float/double conversions on the FP64-bound paths go through fconv.h.
// The polar rotation R, the rhs f, the constraint values C(q_n) and the hinge
// frames are computed in FP64, so the system being refined is the FP64 one.
// All body-space work is done in the body's rest frame: with
// dqb = diag4(R^T) dq, H dq = diag4(R) Hbar dqb (Eq. abd_final).
#include "mabd_mx.cuh"

namespace mabd {

// g = diag4(R^T) sum_k G_kj^T lam_k for body j: a row with point p and world
// direction d contributes s [p; 1] (x) (R^T d) lam_r (s = +1 on body a, -1 on b)
// (HWCVT: multipliers converted with the conversion instruction instead of
// fconv.h's integer path; the final kernel, which is not bound by the FP64
// unit, runs faster that way)
template <typename T, bool XJ, bool HWCVT = false>
__device__ __forceinline__ void gen_force(const DevJoints &J, const DevIncidence &I, int j,
                                          const T R[9], const double *lam, T g[12]) {
  const int K = J.K;
#pragma unroll
  for (int i = 0; i < 12; ++i) g[i] = T(0);
  const int e0 = I.off[j], e1 = I.off[j + 1];
  for (int e = e0; e < e1; ++e) {
    const int k = I.joint[e];
    const int side = I.side[e];
    const int type = J.type[k];
    const T sgn = side == 0 ? T(1) : T(-1);
    T l[5];
#pragma unroll
    for (int r = 0; r < 5; ++r) l[r] = HWCVT ? (T)lam[(size_t)r * K + k] : from_f64<T>(lam[(size_t)r * K + k]);
    const T *p1 = JP<T>::p1(J, side);
    const T *p2 = JP<T>::p2(J, side);
    T F1[3], F2[3], P1[3], P2[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) P1[a] = __ldg(p1 + (size_t)a * K + k);
    T w2 = T(1);        // translation weight of the second point
    bool second = type == 1;
    if (type == 0) {
      F1[0] = l[0];
      F1[1] = l[1];
      F1[2] = l[2];
    } else {
      T RH[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) RH[i] = JP<T>::RH(J)[(size_t)i * K + k];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        F1[a] = RH[a] * l[0] + RH[3 + a] * l[1] + RH[6 + a] * l[2];
        // hinge: rows 3, 4 along R_H's x and z rows; universal: row 3 along
        // a1 (R_U's row 1) at b's point difference l a2, + on b (the
        // negation cancels sgn = -1 below), nothing on a
        F2[a] = (!XJ || type == 1) ? l[3] * RH[a] + l[4] * RH[6 + a] : -l[3] * RH[3 + a];
        P2[a] = __ldg(p2 + (size_t)a * K + k);
      }
      if ((XJ && type == 2)) {
        second = side == 1;
        w2 = T(0);
      }
      if ((XJ && type == 3)) {
        // prismatic: x~, z~ at the anchors, x~, z~ on the axis, z~ off it
        second = true;
        const T *p3 = JP<T>::p3(J, side);
        T F3[3], P3[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          F1[a] = RH[a] * l[0] + RH[6 + a] * l[1];
          F2[a] = RH[a] * l[2] + RH[6 + a] * l[3];
          F3[a] = RH[6 + a] * l[4];
          P3[a] = __ldg(p3 + (size_t)a * K + k);
        }
        T f3[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) f3[a] = sgn * (R[a] * F3[0] + R[3 + a] * F3[1] + R[6 + a] * F3[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          g[a] += P3[0] * f3[a];
          g[3 + a] += P3[1] * f3[a];
          g[6 + a] += P3[2] * f3[a];
          g[9 + a] += f3[a];
        }
      }
    }
    T f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) f[a] = sgn * (R[a] * F1[0] + R[3 + a] * F1[1] + R[6 + a] * F1[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      g[a] += P1[0] * f[a];
      g[3 + a] += P1[1] * f[a];
      g[6 + a] += P1[2] * f[a];
      g[9 + a] += f[a];
    }
    if (second) {
#pragma unroll
      for (int a = 0; a < 3; ++a) f[a] = sgn * (R[a] * F2[0] + R[3 + a] * F2[1] + R[6 + a] * F2[2]);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        g[a] += P2[0] * f[a];
        g[3 + a] += P2[1] * f[a];
        g[6 + a] += P2[2] * f[a];
        g[9 + a] += w2 * f[a];
      }
    }
  }
}

// gen_force for ball and hinge joints in double-float: g = diag4(R^T)
// sum_k G_kj^T lam_k
__device__ __forceinline__ void gen_force_ff(const DevJoints &J, const DevIncidence &I, int j,
                                             const ff R[9], const double *lam, ff g[12]) {
  const int K = J.K;
#pragma unroll
  for (int i = 0; i < 12; ++i) g[i] = ff_make(0.0f);
  auto add_point = [&](const ff F[3], const ff P[3], bool neg) {
    ff f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      f[a] = ff_fma(R[a], F[0], ff_fma(R[3 + a], F[1], ff_mul(R[6 + a], F[2])));
      if (neg) f[a] = ff_neg(f[a]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      g[a] = ff_fma(P[0], f[a], g[a]);
      g[3 + a] = ff_fma(P[1], f[a], g[3 + a]);
      g[6 + a] = ff_fma(P[2], f[a], g[6 + a]);
      g[9 + a] = ff_add(g[9 + a], f[a]);
    }
  };
  const int e0 = I.off[j], e1 = I.off[j + 1];
  for (int e = e0; e < e1; ++e) {
    const int k = I.joint[e];
    const int side = I.side[e];
    const int type = J.type[k];
    const double *p1 = side == 0 ? J.pa1 : J.pb1;
    ff P1[3], l[5], F1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) P1[a] = ff_from(__ldg(p1 + (size_t)a * K + k));
#pragma unroll
    for (int r = 0; r < 3; ++r) l[r] = ff_from(lam[(size_t)r * K + k]);
    if (type == 0) {
      F1[0] = l[0];
      F1[1] = l[1];
      F1[2] = l[2];
      add_point(F1, P1, side == 1);
    } else {
      l[3] = ff_from(lam[(size_t)3 * K + k]);
      l[4] = ff_from(lam[(size_t)4 * K + k]);
      const double *p2 = side == 0 ? J.pa2 : J.pb2;
      ff RH[9], F2[3], P2[3];
#pragma unroll
      for (int i = 0; i < 9; ++i) RH[i] = ff_from(J.RH[(size_t)i * K + k]);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        F1[a] = ff_fma(RH[a], l[0], ff_fma(RH[3 + a], l[1], ff_mul(RH[6 + a], l[2])));
        F2[a] = ff_fma(RH[a], l[3], ff_mul(RH[6 + a], l[4]));
        P2[a] = ff_from(__ldg(p2 + (size_t)a * K + k));
      }
      add_point(F1, P1, side == 1);
      add_point(F2, P2, side == 1);
    }
  }
}

// One thread per body: R = polar(A) and the rest-frame rhs
// fbar = diag4(R^T)(M_A qdot/h + [0; m g]) - [V vec P(R^T A); 0]
// (Sec. 3.3-3.4) in double-float arithmetic (ff.h: ~46 bits; the binary64
// state split with integer instructions; R stored as binary64 and as the
// pair (Rf, Rlo), fbar as the pair (fbh, fbl)), which keeps them off the
// FP64 unit; u = Hbar^{-1} fbar in FP32.
__global__ void __launch_bounds__(128, 5) k_mx_body_prep(DevBodies B, StepParams p, int *status,
                                                      unsigned long long *iters) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= B.M) return;
  const int M = B.M;
  // every load issued before the polar iteration, so that their latency
  // hides behind it
  double qa[9], qv[12], cst[6];
#pragma unroll
  for (int i = 0; i < 9; ++i) qa[i] = B.q[(size_t)i * M + j];
#pragma unroll
  for (int i = 0; i < 12; ++i) qv[i] = B.qd[(size_t)i * M + j];
  cst[0] = ldg(B.sig + j);
  cst[1] = ldg(B.sig + M + j);
  cst[2] = ldg(B.sig + 2 * (size_t)M + j);
  cst[3] = ldg(B.mass + j);
  cst[4] = ldg(B.vmu + j);
  cst[5] = ldg(B.vlam + j);
  const bool fixed = B.fixed[j] != 0;
  ff A[9], R[9];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int r = 0; r < 3; ++r) A[3 * r + c] = ff_from(qa[3 * c + r]);
  int nit = 0;
  int st = polar3_ff(A, R, &nit);
  if (iters) count_add(iters, (unsigned)nit);
  if (st) {
    set_status(status, st);
#pragma unroll
    for (int i = 0; i < 9; ++i) R[i] = ff_make((i % 4 == 0) ? 1.0f : 0.0f);
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    B.R[(size_t)i * M + j] = ff_to(R[i]);
    B.Rf[(size_t)i * M + j] = R[i].h;
    B.Rlo[(size_t)i * M + j] = R[i].l;
  }
  if (fixed) return;  // no unknowns; its rotation may still orient a hinge
  ff qd[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) qd[i] = ff_from(qv[i]);
  ff fb[12];
  fbar_ff(A, R, qd, cst, p, fb);
  float hf[16], ff32[12], u[12];
  load_hinvf(B, j, hf);
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    B.fbh[(size_t)i * M + j] = fb[i].h;
    B.fbl[(size_t)i * M + j] = fb[i].l;
    ff32[i] = fb[i].h;
  }
  hinv_apply_t(hf, ff32, u);
#pragma unroll
  for (int i = 0; i < 12; ++i) B.ubf[(size_t)i * M + j] = u[i];
}

// One thread per joint: C(q_n) and the joint frame in FP64 (Eq. ball / hinge /
// universal / prismatic; hinge axis from body a with a_y >= 0),
// b = G u + C(q_n) with G u in FP32.
template <bool XJ>
__global__ void __launch_bounds__(128, 6) k_mx_joint_prep(DevBodies B, DevJoints J, StepParams p,
                                                       int *status) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= J.K) return;
  const int k = ordered(J.order, t);
  const int K = J.K, M = B.M;
  const int type = J.type[k];
  const int ia = J.ja[k], ib = J.jb[k];
  const uint8_t fl = J.flags[k];
  const int npt = type == 1 ? 2 : ((XJ && type == 3) ? 3 : 1);  // points whose gap is constrained
  double qa[12], qb[12], pa[3][3], pb[3][3];
  load12(B.q, M, ia, qa);
  if (fl & JF_B_BODY) load12(B.q, M, ib, qb);
  load3(J.pa1, K, k, pa[0]);
  load3(J.pb1, K, k, pb[0]);
  if (type == 1 || (XJ && type == 3)) {
    load3(J.pa2, K, k, pa[1]);
    load3(J.pb2, K, k, pb[1]);
  }
  if ((XJ && type == 3)) {
    load3(J.pa3, K, k, pa[2]);
    load3(J.pb3, K, k, pb[2]);
  }
  // gaps of the constrained points (FP64) and their displacements under u (FP32)
  double d[3][3];
  float g[3][3];
  for (int t = 0; t < npt; ++t) {
    gap_of(qa, pa[t], (fl & JF_B_BODY) ? qb : nullptr, pb[t], d[t]);
    g[t][0] = g[t][1] = g[t][2] = 0.f;
  }
  for (int sd = 0; sd < 2; ++sd) {
    if (!(fl & (sd == 0 ? JF_A_FREE : JF_B_FREE))) continue;
    const int i = sd == 0 ? ia : ib;
    float R[9], u[12];
    load_Rf(B, i, R);
#pragma unroll
    for (int c = 0; c < 12; ++c) u[c] = B.ubf[(size_t)c * M + i];
    for (int t = 0; t < npt; ++t) {
      float pf[3];
      const float *src = sd == 0 ? (t == 0 ? J.pa1f : (t == 1 ? J.pa2f : J.pa3f))
                                 : (t == 0 ? J.pb1f : (t == 1 ? J.pb2f : J.pb3f));
      load3f(src, K, k, pf);
      float x[3];
      disp_at(R, u, pf, x);
#pragma unroll
      for (int a = 0; a < 3; ++a) g[t][a] += sd == 0 ? x[a] : -x[a];
    }
  }
  const double rr = p.residual_rhs ? 1.0 : 0.0;
  if ((XJ && type == 3)) {
    // prismatic (Sec. 4.5): x~, z~ of the anchor and on-axis gaps, z~ of the
    // off-axis gap, in R_P attached to a
    double uax[3], ca[3], Ra[9], RP[9];
    load3(J.ua, K, k, uax);
    load_R(B.R, M, ia, Ra);
#pragma unroll
    for (int a = 0; a < 3; ++a) ca[a] = pa[2][a] - pa[0][a];
    prismatic_frame(Ra, uax, ca, RP);
    float RPf[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) RPf[i] = d2f(RP[i]);
    const int tpt[5] = {0, 0, 1, 1, 2};
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      const int o = (r == 0 || r == 2) ? 0 : 6, q = tpt[r];
      const double c = RP[o] * d[q][0] + RP[o + 1] * d[q][1] + RP[o + 2] * d[q][2];
      const float e = RPf[o] * g[q][0] + RPf[o + 1] * g[q][1] + RPf[o + 2] * g[q][2];
      J.c[(size_t)r * K + k] = c;
      J.b[(size_t)r * K + k] = f2d(e) + rr * c;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      J.RH[(size_t)i * K + k] = RP[i];
      J.RHf[(size_t)i * K + k] = RPf[i];
    }
    return;
  }
  if (type == 0) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      J.c[(size_t)r * K + k] = d[0][r];
      J.b[(size_t)r * K + k] = f2d(g[0][r]) + rr * d[0][r];
    }
    return;
  }
  if ((XJ && type == 2)) {
    // universal (Sec. 4.4): ball rows in R_U, row 3 = a1 . A_b (l a2) on b alone
    double uax[3], vb[3], Ra[9], Rb[9], RU[9], Ab[9], xb[3], c1[3];
    load3(J.ua, K, k, uax);
    load3(J.pb2, K, k, vb);
    load_R(B.R, M, ia, Ra);
    load_R(B.R, M, ib, Rb);
    universal_frame(Ra, uax, Rb, vb, RU);
    A_from_q(qb, Ab);
    mv3(Ab, vb, xb);
    mv3(RU, d[0], c1);
    float RUf[9], gb3[3] = {0.f, 0.f, 0.f}, e1[3];
#pragma unroll
    for (int i = 0; i < 9; ++i) RUf[i] = d2f(RU[i]);
    if (fl & JF_B_FREE) {
      float Rbf[9], u[12], vbf[3], l[3];
      load_Rf(B, ib, Rbf);
#pragma unroll
      for (int c = 0; c < 12; ++c) u[c] = B.ubf[(size_t)c * M + ib];
      load3f(J.pb2f, K, k, vbf);
#pragma unroll
      for (int a = 0; a < 3; ++a) l[a] = u[a] * vbf[0] + u[3 + a] * vbf[1] + u[6 + a] * vbf[2];
      mv3(Rbf, l, gb3);
    }
    mv3(RUf, g[0], e1);
    const double c3 = RU[3] * xb[0] + RU[4] * xb[1] + RU[5] * xb[2];
    const float e3 = RUf[3] * gb3[0] + RUf[4] * gb3[1] + RUf[5] * gb3[2];
    const double cc[4] = {c1[0], c1[1], c1[2], c3};
    const float gg[4] = {e1[0], e1[1], e1[2], e3};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      J.c[(size_t)r * K + k] = cc[r];
      J.b[(size_t)r * K + k] = f2d(gg[r]) + rr * cc[r];
    }
    J.c[(size_t)4 * K + k] = 0.0;
    J.b[(size_t)4 * K + k] = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      J.RH[(size_t)i * K + k] = RU[i];
      J.RHf[(size_t)i * K + k] = RUf[i];
    }
    return;
  }
  double uax[3], a[3], Ra[9], RH[9];
  load3(J.ua, K, k, uax);
  load_R(B.R, M, ia, Ra);
  mv3(Ra, uax, a);
  {
    const double n = rsqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    const double sgn = a[1] < 0.0 ? -n : n;
    a[0] *= sgn; a[1] *= sgn; a[2] *= sgn;
  }
  hinge_frame(a, RH);
  float RHf[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) RHf[i] = d2f(RH[i]);
  double c1[3], c2[3];
  float e1[3], e2[3];
  mv3(RH, d[0], c1);
  mv3(RH, d[1], c2);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    e1[r] = RHf[3 * r] * g[0][0] + RHf[3 * r + 1] * g[0][1] + RHf[3 * r + 2] * g[0][2];
    e2[r] = RHf[3 * r] * g[1][0] + RHf[3 * r + 1] * g[1][1] + RHf[3 * r + 2] * g[1][2];
  }
  const double cc[5] = {c1[0], c1[1], c1[2], c2[0], c2[2]};
  const float gg[5] = {e1[0], e1[1], e1[2], e2[0], e2[2]};
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    J.c[(size_t)r * K + k] = cc[r];
    J.b[(size_t)r * K + k] = f2d(gg[r]) + rr * cc[r];
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    J.RH[(size_t)i * K + k] = RH[i];
    J.RHf[(size_t)i * K + k] = RHf[i];
  }
}

// One thread per body, start of a correction sweep.  First chain sweep:
// dqb = u - Hbar^{-1} g(lambda) in FP32 (back-propagation of the approximate
// solve); later chain sweeps: dqb += z - Hbar^{-1} g(dlambda) (the previous
// correction); tree: dqb as the elimination left it.  Then the primal residual
// rb = fbar - Hbar dqb - g(lambda) in double-float (the FP64 system's
// residual to ~46 bits) and the correction's unconstrained solve
// z = Hbar^{-1} rb in FP32 (kept in ubf).
template <int MODE, bool XJ>
__global__ void __launch_bounds__(128, 5) k_mx_res_body(DevBodies B, DevJoints J, DevIncidence I,
                                                     StepParams p) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B.M) return;
  const int j = ordered(B.order, t);
  if (B.fixed[j]) return;
  const int M = B.M;
  float hf[16], uf[12], w[12], gf[12];
  load_hinvf(B, j, hf);
#pragma unroll
  for (int i = 0; i < 12; ++i) uf[i] = B.ubf[(size_t)i * M + j];
  ff R[9], g[12], dq[12];
#pragma unroll
  for (int i = 0; i < 9; ++i) R[i] = ff{B.Rf[(size_t)i * M + j], B.Rlo[(size_t)i * M + j]};
  if (XJ) {
    // universal and prismatic joints: the FP64 generalized force
    double Rd[9], g64[12];
    load_R(B.R, M, j, Rd);
    gen_force<double, XJ>(J, I, j, Rd, J.lambda, g64);
#pragma unroll
    for (int i = 0; i < 12; ++i) g[i] = ff_from(g64[i]);
  } else {
    gen_force_ff(J, I, j, R, J.lambda, g);
  }
  if (MODE == MX_FROM_U) {
#pragma unroll
    for (int i = 0; i < 12; ++i) gf[i] = g[i].h;
    hinv_apply_t(hf, gf, w);
#pragma unroll
    for (int i = 0; i < 12; ++i) dq[i] = ff_make(uf[i] - w[i]);
  } else if (MODE == MX_FROM_CORRECTION) {
    float Rf[9];
    load_Rf(B, j, Rf);
    gen_force<float, XJ>(J, I, j, Rf, J.dlam, gf);
    hinv_apply_t(hf, gf, w);
#pragma unroll
    for (int i = 0; i < 12; ++i) dq[i] = ff_add(ff_from(B.dqb[(size_t)i * M + j]), ff_make(uf[i] - w[i]));
  } else {
#pragma unroll
    for (int i = 0; i < 12; ++i) dq[i] = ff_from(B.dqb[(size_t)i * M + j]);
  }
  const ff s[3] = {ff_from(ldg(B.sig + j)), ff_from(ldg(B.sig + M + j)), ff_from(ldg(B.sig + 2 * (size_t)M + j))};
  const ff ih = ff_from(p.inv_h);
  ff hq[12];
  hbar_apply_ff(s, ff_from(ldg(B.mass + j)), ff_from(ldg(B.vmu + j)), ff_from(ldg(B.vlam + j)), ff_mul(ih, ih),
                dq, hq);
  float rf[12], z[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    const ff fb = ff{B.fbh[(size_t)i * M + j], B.fbl[(size_t)i * M + j]};
    rf[i] = ff_sub(ff_sub(fb, hq[i]), g[i]).h;
  }
  hinv_apply_t(hf, rf, z);
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    if (MODE == MX_FROM_U) B.dqb[(size_t)i * M + j] = f2d(dq[i].h);
    else if (MODE == MX_FROM_CORRECTION) B.dqb[(size_t)i * M + j] = ff_to(dq[i]);
    B.ubf[(size_t)i * M + j] = z[i];
  }
}

// One thread per joint: correction rhs b = G z + (C(q_n) + G dq), the
// bracket (the FP64 dual residual, negated) in FP64 and G z in FP32; the
// largest |C + G dq| goes to *maxbit when it is given.  With the printed zero
// bottom rhs (residual_rhs = 0) the constraint is G dq = 0 and C drops out.
template <bool XJ>
__global__ void __launch_bounds__(128, 6) k_mx_res_joint(DevBodies B, DevJoints J, StepParams p,
                                                      unsigned long long *maxbit, bool add_gz) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double worst = 0.0;
  if (t < J.K) {
    const int k = ordered(J.order, t);
    const int K = J.K, M = B.M;
    const int type = J.type[k];
    const int ia = J.ja[k], ib = J.jb[k];
    const uint8_t fl = J.flags[k];
    const int npt = type == 1 ? 2 : ((XJ && type == 3) ? 3 : 1);
    double pa[3][3], pb[3][3], d[3][3], d3[3] = {0.0, 0.0, 0.0};
    float e[3][3], e3[3] = {0.f, 0.f, 0.f};
    load3(J.pa1, K, k, pa[0]);
    load3(J.pb1, K, k, pb[0]);
    if (type == 1 || (XJ && type == 3)) {
      load3(J.pa2, K, k, pa[1]);
      load3(J.pb2, K, k, pb[1]);
    }
    if ((XJ && type == 3)) {
      load3(J.pa3, K, k, pa[2]);
      load3(J.pb3, K, k, pb[2]);
    }
    for (int t = 0; t < 3; ++t)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        d[t][a] = 0.0;
        e[t][a] = 0.f;
      }
    for (int sd = 0; sd < 2; ++sd) {
      if (!(fl & (sd == 0 ? JF_A_FREE : JF_B_FREE))) continue;
      const int i = sd == 0 ? ia : ib;
      double R[9], x[12];
      float Rf[9], z[12];
      load_R(B.R, M, i, R);
      load12(B.dqb, M, i, x);
      load_Rf(B, i, Rf);
#pragma unroll
      for (int c = 0; c < 12; ++c) z[c] = B.ubf[(size_t)c * M + i];
      for (int t = 0; t < npt; ++t) {
        const double *pp = sd == 0 ? pa[t] : pb[t];
        float pf[3];
        const float *src = sd == 0 ? (t == 0 ? J.pa1f : (t == 1 ? J.pa2f : J.pa3f))
                                   : (t == 0 ? J.pb1f : (t == 1 ? J.pb2f : J.pb3f));
        load3f(src, K, k, pf);
        double xd[3];
        float xf[3];
        disp_at(R, x, pp, xd);
        disp_at(Rf, z, pf, xf);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          d[t][a] += sd == 0 ? xd[a] : -xd[a];
          e[t][a] += sd == 0 ? xf[a] : -xf[a];
        }
      }
      if ((XJ && type == 2) && sd == 1) {
        // universal row 3: b's axis vector l a2 moved by dq (FP64) and by z (FP32)
        double vb[3], l[3];
        float vbf[3], lf[3];
        load3(J.pb2, K, k, vb);
        load3f(J.pb2f, K, k, vbf);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          l[a] = x[a] * vb[0] + x[3 + a] * vb[1] + x[6 + a] * vb[2];
          lf[a] = z[a] * vbf[0] + z[3 + a] * vbf[1] + z[6 + a] * vbf[2];
        }
        mv3(R, l, d3);
        mv3(Rf, lf, e3);
      }
    }
    double v[5];
    float w[5];
    int C = 3;
    if (type == 0) {
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        v[r] = d[0][r];
        w[r] = e[0][r];
      }
    } else if ((XJ && type == 2)) {
      C = 4;
      double RU[9];
      float RUf[9];
      load_R(J.RH, K, k, RU);
#pragma unroll
      for (int i = 0; i < 9; ++i) RUf[i] = J.RHf[(size_t)i * K + k];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        v[r] = RU[3 * r] * d[0][0] + RU[3 * r + 1] * d[0][1] + RU[3 * r + 2] * d[0][2];
        w[r] = RUf[3 * r] * e[0][0] + RUf[3 * r + 1] * e[0][1] + RUf[3 * r + 2] * e[0][2];
      }
      v[3] = RU[3] * d3[0] + RU[4] * d3[1] + RU[5] * d3[2];
      w[3] = RUf[3] * e3[0] + RUf[4] * e3[1] + RUf[5] * e3[2];
    } else if ((XJ && type == 3)) {
      // prismatic: x~, z~ at the anchors, x~, z~ on the axis, z~ off it
      C = 5;
      double RP[9];
      float RPf[9];
      load_R(J.RH, K, k, RP);
#pragma unroll
      for (int i = 0; i < 9; ++i) RPf[i] = J.RHf[(size_t)i * K + k];
      const int tpt[5] = {0, 0, 1, 1, 2};
#pragma unroll
      for (int r = 0; r < 5; ++r) {
        const int o = (r == 0 || r == 2) ? 0 : 6, q = tpt[r];
        v[r] = RP[o] * d[q][0] + RP[o + 1] * d[q][1] + RP[o + 2] * d[q][2];
        w[r] = RPf[o] * e[q][0] + RPf[o + 1] * e[q][1] + RPf[o + 2] * e[q][2];
      }
    } else {
      C = 5;
      double RH[9];
      load_R(J.RH, K, k, RH);
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        v[r] = RH[3 * r] * d[0][0] + RH[3 * r + 1] * d[0][1] + RH[3 * r + 2] * d[0][2];
      }
      float RHf[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) RHf[i] = J.RHf[(size_t)i * K + k];
#pragma unroll
      for (int r = 0; r < 3; ++r)
        w[r] = RHf[3 * r] * e[0][0] + RHf[3 * r + 1] * e[0][1] + RHf[3 * r + 2] * e[0][2];
      v[3] = RH[0] * d[1][0] + RH[1] * d[1][1] + RH[2] * d[1][2];
      v[4] = RH[6] * d[1][0] + RH[7] * d[1][1] + RH[8] * d[1][2];
      w[3] = RHf[0] * e[1][0] + RHf[1] * e[1][1] + RHf[2] * e[1][2];
      w[4] = RHf[6] * e[1][0] + RHf[7] * e[1][1] + RHf[8] * e[1][2];
    }
    for (int r = 0; r < C; ++r) {
      const double res = (p.residual_rhs ? J.c[(size_t)r * K + k] : 0.0) + v[r];
      worst = fmax(worst, fabs(res));
      J.b[(size_t)r * K + k] = add_gz ? f2d(w[r]) + res : res;
    }
  }
  if (maxbit) {
    for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(maxbit, worst);
  }
}

// One thread per body, end of the step.  Chain: dqb (+)= z - Hbar^{-1} g(l)
// with l = lambda after the approximate solve alone (MX_FROM_U: z is u and dqb
// starts at zero), else l = the last correction dlambda; tree (MX_FROM_DQB):
// dqb as the eliminations left it.  Then dq = diag4(R) dqb, q += dq,
// qdot = dq / h (implicit Euler, Sec. 3.4).
template <bool XJ>
__global__ void __launch_bounds__(128, 6) k_mx_final(DevBodies B, DevJoints J, DevIncidence I,
                                                  StepParams p, int mode) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B.M) return;
  const int j = ordered(B.order, t);
  if (B.fixed[j]) return;
  const int M = B.M;
  double R[9];
  load_R(B.R, M, j, R);
  double x[12];
  if (mode == MX_FROM_DQB) {
    load12(B.dqb, M, j, x);
  } else {
    const bool from_u = mode == MX_FROM_U;
    float Rf[9], hf[16], gf[12], w[12];
    load_Rf(B, j, Rf);
    load_hinvf(B, j, hf);
    gen_force<float, XJ, true>(J, I, j, Rf, from_u ? J.lambda : J.dlam, gf);
    hinv_apply_t(hf, gf, w);
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      const double base = from_u ? 0.0 : B.dqb[(size_t)i * M + j];
      x[i] = base + (double)(B.ubf[(size_t)i * M + j] - w[i]);
    }
  }
#pragma unroll
  for (int blk = 0; blk < 4; ++blk) {
    double dq[3];
    mv3(R, x + 3 * blk, dq);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const size_t o = (size_t)(3 * blk + a) * M + j;
      B.q[o] += dq[a];
      B.qd[o] = dq[a] * p.inv_h;
    }
  }
}

static inline int nblk(int n, int t) { return (n + t - 1) / t; }

void launch_mx_body_prep(const DevBodies &B, const StepParams &p, int *status, cudaStream_t s,
                         unsigned long long *iters) {
  if (B.M > 0) k_mx_body_prep<<<nblk(B.M, 128), 128, 0, s>>>(B, p, status, iters);
}

void launch_mx_joint_prep(const DevBodies &B, const DevJoints &J, const StepParams &p, int *status,
                          cudaStream_t s) {
  if (J.K == 0) return;
  if (J.xj) k_mx_joint_prep<true><<<nblk(J.K, 128), 128, 0, s>>>(B, J, p, status);
  else k_mx_joint_prep<false><<<nblk(J.K, 128), 128, 0, s>>>(B, J, p, status);
}

void launch_mx_res_body(const DevBodies &B, const DevJoints &J, const DevIncidence &I,
                        const StepParams &p, int mode, cudaStream_t s) {
  if (B.M <= 0) return;
  const dim3 g(nblk(B.M, 128));
  if (J.xj) {
    if (mode == MX_FROM_U) k_mx_res_body<MX_FROM_U, true><<<g, 128, 0, s>>>(B, J, I, p);
    else if (mode == MX_FROM_CORRECTION) k_mx_res_body<MX_FROM_CORRECTION, true><<<g, 128, 0, s>>>(B, J, I, p);
    else k_mx_res_body<MX_FROM_DQB, true><<<g, 128, 0, s>>>(B, J, I, p);
  } else {
    if (mode == MX_FROM_U) k_mx_res_body<MX_FROM_U, false><<<g, 128, 0, s>>>(B, J, I, p);
    else if (mode == MX_FROM_CORRECTION) k_mx_res_body<MX_FROM_CORRECTION, false><<<g, 128, 0, s>>>(B, J, I, p);
    else k_mx_res_body<MX_FROM_DQB, false><<<g, 128, 0, s>>>(B, J, I, p);
  }
}

void launch_mx_res_joint(const DevBodies &B, const DevJoints &J, const StepParams &p,
                         unsigned long long *maxbit, cudaStream_t s, bool add_gz) {
  if (J.K == 0) return;
  if (J.xj) k_mx_res_joint<true><<<nblk(J.K, 128), 128, 0, s>>>(B, J, p, maxbit, add_gz);
  else k_mx_res_joint<false><<<nblk(J.K, 128), 128, 0, s>>>(B, J, p, maxbit, add_gz);
}

void launch_mx_final(const DevBodies &B, const DevJoints &J, const DevIncidence &I,
                     const StepParams &p, int mode, cudaStream_t s) {
  if (B.M == 0) return;
  if (J.xj) k_mx_final<true><<<nblk(B.M, 128), 128, 0, s>>>(B, J, I, p, mode);
  else k_mx_final<false><<<nblk(B.M, 128), 128, 0, s>>>(B, J, I, p, mode);
}

}  // namespace mabd
