// Tree path of one M-ABD step, Sec. 5.3 (Alg. 2, Eq. module3-kkt), read as
// the exact constraint-row elimination in body space, templated on the
// elimination's type S (double: the FP64 form; float: the FP32 elimination of
// the mixed form, whose right-hand side and outputs DevTreeT names):
//   upward (deepest level first), body j with parent joint rows G (on j) and
//   P (on the parent):
//     Hhat_j = Hbar_j + sum_children U_i U_i^T,  fhat_j = fbar_j - sum_children v_i
//     y = Hhat_j^{-1} fhat_j, X = Hhat_j^{-1} G^T, D = G X = L_D L_D^T,
//     e = G y + C(q_n),  U = P^T L_D^{-T},  v = P^T D^{-1} e   (to the parent)
//   downward (roots first):
//     lambda = D^{-1}(e + P dq_parent),  dq_j = y - X lambda.
// Everything of body j is kept in its rest frame (rows s [p;1] (x) R_j^T d).
//
// Every body of the upward pass is eliminated by a group of 16 lanes, lane r
// < 12 holding row r of the body's 12 x 12 system.  A leaf applies the
// structured Hbar^{-1} (at most three entries per row, gathered by
// shuffles); a body with children factors its dense Hhat by a right-looking
// Cholesky that carries the right-hand sides along (see up_body).  The code
// keeps its loops rolled: a level with a handful of bodies runs the same few
// kilobytes of instructions again and again instead of fetching a long
// unrolled sequence once, which is what bounds a narrow level's latency.
// Ball joints are padded to five rows (zero rows, unit pivots), so one
// instantiation serves both joint types.  The level-scheduled launches and a
// persistent kernel (one block per tree) are chosen by the tuner in
// mabd_api.cpp.
#include "mabd_device.cuh"

namespace mabd {

__device__ __forceinline__ int p12(int r, int c) { return r * (r + 1) / 2 + c; }  // r >= c

// an FP64 body constant in the elimination's type S
template <typename S>
__device__ __forceinline__ S ldgs(const double *p) { return from_f64<S>(__ldg(p)); }

// the body inputs of the elimination in its type: rotation, structured
// Hbar^{-1} and the unconstrained rest-frame solve ubar = Hbar^{-1} fbar
template <typename S> struct TB;
template <> struct TB<double> {
  __device__ static const double *R(const DevBodies &B) { return B.R; }
  __device__ static const double *hinv(const DevBodies &B) { return B.hinv; }
  __device__ static const double *ubar(const DevBodies &B) { return B.ubar; }
};
template <> struct TB<float> {
  __device__ static const float *R(const DevBodies &B) { return B.Rf; }
  __device__ static const float *hinv(const DevBodies &B) { return B.hinvf; }
  __device__ static const float *ubar(const DevBodies &B) { return B.ubf; }
};

// a multiplier of the solve: to T.lam (FP64) and, when given, added to T.lam_acc
template <typename S>
__device__ __forceinline__ void put_lambda(const DevTreeT<S> &T, size_t o, S v) {
  const double v64 = to_f64(v);
  T.lam[o] = v64;
  if (T.lam_acc) T.lam_acc[o] += v64;
}

constexpr int RMAX = 10;  // rows eliminated at a root (two one-sided joints)
constexpr int NJ = 5;     // rows of a parent joint as eliminated (ball joints padded)
constexpr int GL = 16;    // lanes per body
constexpr int GSC = 144;  // per-group scratch (S values): the Cholesky factor L, 12 x 12

template <typename S>
__device__ __forceinline__ S gshfl(unsigned m, S v, int src) { return __shfl_sync(m, v, src, GL); }
template <typename S>
__device__ __forceinline__ S gxor(unsigned m, S v, int o) { return __shfl_xor_sync(m, v, o, GL); }

// entry (r, c) of the dense Hbar of Sec. 3: the 3x3 block of A's diagonal
// entries (rows 0, 4, 8), the transpose pairs (1, 3), (2, 6), (5, 7) and the
// translation; r and c may be run-time values (the tests become selects)
template <typename S>
__device__ __forceinline__ S hbar_rc(int r, int c, const S s[3], S vm, S vl, S m, S ih2) {
  const bool dr = (r == 0 || r == 4 || r == 8), dc = (c == 0 || c == 4 || c == 8);
  if (r == c) {
    if (r >= 9) return m * ih2;
    const S sd = r < 3 ? s[0] : (r < 6 ? s[1] : s[2]);
    return sd * ih2 + vm + (dr ? vm + vl : S(0));
  }
  if (dr && dc) return vl;
  const int a = r < c ? r : c, bq = r < c ? c : r;
  if ((a == 1 && bq == 3) || (a == 2 && bq == 6) || (a == 5 && bq == 7)) return vm;
  return S(0);
}

// (Hbar x)_l for the structured Hbar of a body: row l's (up to three)
// non-zeros against x gathered from the lanes (x_c on lane c)
template <typename S>
__device__ __forceinline__ S hbar_row_apply(int l, const S s[3], S vm, S vl, S m, S ih2, S xl, unsigned gm) {
  const S x0 = gshfl(gm, xl, 0), x4 = gshfl(gm, xl, 4), x8 = gshfl(gm, xl, 8);
  const int pr = l == 1 ? 3 : l == 3 ? 1 : l == 2 ? 6 : l == 6 ? 2 : l == 5 ? 7 : l == 7 ? 5 : l;
  const S xp = gshfl(gm, xl, pr & 15);
  if (l >= 9) return m * ih2 * xl;
  if (l == 0 || l == 4 || l == 8) return hbar_rc(l, l, s, vm, vl, m, ih2) * xl + vl * (x0 + x4 + x8 - xl);
  return hbar_rc(l, l, s, vm, vl, m, ih2) * xl + vm * xp;
}

// Row l of the structured Hbar^{-1} (layout of hinv_apply): the h[16] slots
// ih[q] (-1: none) of its entries and their columns ic[q]
__device__ __forceinline__ void hinv_row(int l, int ih[3], int ic[3]) {
  ih[0] = ih[1] = ih[2] = -1;
  ic[0] = ic[1] = ic[2] = l & 15;
  if (l >= 12) return;
  if (l >= 9) {
    ih[0] = 0;
  } else if (l == 0 || l == 4 || l == 8) {
    ic[0] = 0; ic[1] = 4; ic[2] = 8;
    ih[0] = l == 0 ? 1 : (l == 4 ? 2 : 3);
    ih[1] = l == 0 ? 2 : (l == 4 ? 4 : 5);
    ih[2] = l == 0 ? 3 : (l == 4 ? 5 : 6);
  } else {
    // pairs (1, 3) -> h7..9, (2, 6) -> h10..12, (5, 7) -> h13..15
    const int lo = (l == 1 || l == 3) ? 1 : ((l == 2 || l == 6) ? 2 : 5);
    const int hi = lo == 1 ? 3 : (lo == 2 ? 6 : 7);
    const int base = lo == 1 ? 7 : (lo == 2 ? 10 : 13);
    ic[0] = lo; ic[1] = hi;
    ih[0] = l == lo ? base : base + 1;
    ih[1] = l == lo ? base + 1 : base + 2;
  }
}

// MABD_JACOBIAN_FULL: lane l's entry of the frame term of row r on the
// joint's body a, [qh_r]x on the 3x3 block: +qh_0 at 5, -qh_0 at 7, +qh_1
// at 6, -qh_1 at 2, +qh_2 at 1, -qh_2 at 3 (out of line: the frozen-frame
// path keeps its registers)
__device__ __noinline__ double full_lane_term(const double *qf, int K, int k, int l, int r) {
  const int ax = (l == 5 || l == 7) ? 0 : ((l == 2 || l == 6) ? 1 : ((l == 1 || l == 3) ? 2 : -1));
  if (ax < 0) return 0.0;
  const double v = __ldg(qf + (size_t)(3 * r + ax) * K + k);
  return (l == 5 || l == 6 || l == 1) ? v : -v;
}

// Lane l's entries of the rows of joint k on the body with rotation R that
// is its side `side` (rest frame, Sec. 5.1: s [p; 1] (x) R^T d): Rc = column
// l % 3 of R.  Ball rows (3) are followed by two zero rows.  Returns C.
template <typename S>
__device__ __forceinline__ int lane_rows(const DevJoints &J, int k, int side, const S Rc[3], int l, S w[NJ]) {
  const int K = J.K;
  const int type = J.type[k];
  const S sg = side == 0 ? S(1) : S(-1);
  const int blk = l / 3;
  const S p1 = blk < 3 ? __ldg(JP<S>::p1(J, side) + (size_t)blk * K + k) : S(1);
  if (type == 0) {
    w[0] = sg * p1 * Rc[0];
    w[1] = sg * p1 * Rc[1];
    w[2] = sg * p1 * Rc[2];
    w[3] = w[4] = S(0);
    return 3;
  }
  // hinge: rows 0-2 are R_H's rows at the first point, rows 3 and 4 its x
  // and z rows at the second (Eq. hinge)
  const S p2 = blk < 3 ? __ldg(JP<S>::p2(J, side) + (size_t)blk * K + k) : S(1);
  S g[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const S *RH = JP<S>::RH(J) + (size_t)(3 * r) * K + k;
    g[r] = Rc[0] * __ldg(RH) + Rc[1] * __ldg(RH + K) + Rc[2] * __ldg(RH + 2 * (size_t)K);
  }
  w[0] = sg * p1 * g[0];
  w[1] = sg * p1 * g[1];
  w[2] = sg * p1 * g[2];
  w[3] = sg * p2 * g[0];
  w[4] = sg * p2 * g[2];
  if constexpr (sizeof(S) == 8) {
    if (J.qf && side == 0)  // MABD_JACOBIAN_FULL (FP64 form only)
#pragma unroll
      for (int r = 0; r < 5; ++r) w[r] += full_lane_term(J.qf, K, k, l, r);
  }
  return 5;
}

// column l % 3 of body j's rotation (R row-major)
template <typename S>
__device__ __forceinline__ void rot_col(const DevBodies &B, int j, int l, S Rc[3]) {
  const S *R = TB<S>::R(B);
  const int a = l % 3;
#pragma unroll
  for (int i = 0; i < 3; ++i) Rc[i] = R[(size_t)(3 * i + a) * B.M + j];
}

// Upward pass of body j by a lane group (lane l of mask gm, sc the group's
// scratch): N rows are eliminated, the parent joint's (N = NJ) or a root's
// one-sided joints (ROOT, N = RMAX, unused rows padded).  Writes X, y, L_D, e
// (or the root's rX, rLD, re) and, below a root, U and v for the parent.
template <typename S, int N, bool ROOT>
__device__ __noinline__ void up_body(const DevBodies &B, const DevJoints &J, const DevTreeT<S> &T, int j,
                                     const StepParams &p, int *status, int l, unsigned gm, S *sc) {
  constexpr int NR = 1 + N;  // right-hand sides of a body with children: f, then the rows
  constexpr int ND = N * (N + 1) / 2;
  const int M = B.M, K = J.K;
  const bool act = l < 12;
  const int nch = T.ccount[j];
  // the eliminated rows: lane l's entry of each (rest frame)
  int ks[2] = {-1, -1}, cs[2] = {0, 0};
  const int rid = ROOT ? T.root_id[j] : -1;
  S Rc[3];
  rot_col(B, j, l, Rc);
  S b[NR];
  if constexpr (!ROOT) {
    ks[0] = T.pjoint[j];
    S w[NJ];
    cs[0] = lane_rows(J, ks[0], T.pside[j], Rc, l, w);
#pragma unroll
    for (int t = 0; t < N; ++t) b[1 + t] = act ? w[t] : S(0);
  } else {
#pragma unroll
    for (int t = 0; t < N; ++t) b[1 + t] = S(0);
    for (int q = 0; q < 2; ++q) {
      ks[q] = T.root_joint[(size_t)q * T.nroots + rid];
      if (ks[q] < 0) continue;
      S w[NJ];
      cs[q] = lane_rows(J, ks[q], T.root_side[(size_t)q * T.nroots + rid], Rc, l, w);
      const int off = q == 0 ? 0 : cs[0];
#pragma unroll
      for (int t = 0; t < N; ++t)
#pragma unroll
        for (int s = 0; s < NJ; ++s)
          if (act && t - off == s && s < cs[q]) b[1 + t] = w[s];
    }
  }
  const int nrow = cs[0] + cs[1];
  // partial sums of D and e over the lanes
  S D[ND], ev[N];
  S y;
  if (nch == 0) {
    // structured Hbar^{-1}: X(l, t) = sum_q h[ih_q] w_t(ic_q), y = ubar
    int ih[3], ic[3];
    hinv_row(l, ih, ic);
    S hc[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) hc[q] = ih[q] >= 0 ? TB<S>::hinv(B)[(size_t)ih[q] * M + j] : S(0);
    y = act ? TB<S>::ubar(B)[(size_t)l * M + j] : S(0);
    S X[N];
#pragma unroll
    for (int t = 0; t < N; ++t) {
      S v = S(0);
#pragma unroll
      for (int q = 0; q < 3; ++q) v += hc[q] * gshfl(gm, b[1 + t], ic[q]);
      X[t] = v;
    }
#pragma unroll
    for (int r = 0; r < N; ++r) {
      ev[r] = b[1 + r] * y;
#pragma unroll
      for (int t = 0; t <= r; ++t) D[p12(r, t)] = b[1 + r] * X[t];
    }
#pragma unroll
    for (int t = 0; t < N; ++t) b[1 + t] = X[t];
    b[0] = y;
  } else {
    // row l of Hhat = Hbar + sum_children U U^T, f_l = (Hbar ubar - sum_children v)_l
    const S ih2 = from_f64<S>(p.inv_h * p.inv_h);
    const S s3[3] = {ldgs<S>(B.sig + j), ldgs<S>(B.sig + M + j), ldgs<S>(B.sig + 2 * (size_t)M + j)};
    const S vm = ldgs<S>(B.vmu + j), vl = ldgs<S>(B.vlam + j), m = ldgs<S>(B.mass + j);
    const S ub = act ? TB<S>::ubar(B)[(size_t)l * M + j] : S(0);
    S f = hbar_row_apply(l, s3, vm, vl, m, ih2, ub, gm);
    S h[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) h[q] = act ? hbar_rc(l, q, s3, vm, vl, m, ih2) : S(0);
    const int c0 = T.cfirst[j];
#pragma unroll 1
    for (int c = c0; c < c0 + nch; ++c) {
      // the child's five rows issued together; a ball joint's rows 3 and 4
      // are exact zeros (padding), so all five are added without looking up
      // the child's joint type (one dependent load round fewer)
      S u[NJ];
#pragma unroll
      for (int t = 0; t < NJ; ++t) u[t] = act ? T.U[(size_t)(NJ * l + t) * M + c] : S(0);
      if (act) f -= T.v[(size_t)l * M + c];
#pragma unroll
      for (int t = 0; t < NJ; ++t)
#pragma unroll
        for (int q = 0; q < 12; ++q) h[q] += u[t] * gshfl(gm, u[t], q);
    }
    b[0] = act ? f : S(0);
    // right-looking Cholesky (reciprocal diagonal) carrying the right-hand
    // sides: column c of the working matrix is always h[0] (the rows shift
    // left after each step); L goes to the scratch row by row
    bool ok = true;
    __syncwarp(gm);  // the scratch may still be read for the group's previous body
#pragma unroll 1
    for (int c = 0; c < 12; ++c) {
      S piv = gshfl(gm, h[0], c);
      if (!(piv > S(0))) {
        ok = false;
        piv = S(1);
      }
      const S id = rsq(piv);
      const S lc = l == c ? id : h[0] * id;  // lane c: 1 / L(c, c); below: L(l, c)
      if (act && l >= c) sc[l * 12 + c] = lc;
      if (l == c) {
#pragma unroll
        for (int k = 0; k < NR; ++k) b[k] *= id;
      }
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        const S zc = gshfl(gm, b[k], c);
        if (l > c) b[k] -= lc * zc;
      }
#pragma unroll
      for (int q = 1; q < 12; ++q) {
        const int cq = c + q;
        const S lq = gshfl(gm, lc, cq & 15);
        h[q - 1] = (l >= cq && cq < 12) ? h[q] - lc * lq : h[q];
      }
      h[11] = S(0);
    }
    if (!ok && l == 0) set_status(status, ST_NOT_SPD);
    // D = Z_W^T Z_W and e = Z_W^T z_f with Z = L^{-1} [f W]
#pragma unroll
    for (int r = 0; r < N; ++r) {
      ev[r] = b[1 + r] * b[0];
#pragma unroll
      for (int t = 0; t <= r; ++t) D[p12(r, t)] = b[1 + r] * b[1 + t];
    }
    // backward sweep with L^T: y and X
    __syncwarp(gm);
    const S idr = act ? sc[l * 12 + l] : S(1);
#pragma unroll 1
    for (int i = 11; i >= 0; --i) {
      if (l == i) {
#pragma unroll
        for (int k = 0; k < NR; ++k) b[k] *= idr;
      }
      const S li = (act && l < i) ? sc[i * 12 + l] : S(0);  // L(i, l)
#pragma unroll
      for (int k = 0; k < NR; ++k) b[k] -= li * gshfl(gm, b[k], i);
    }
    y = b[0];
  }
  // sums over the group
#pragma unroll 1
  for (int o = GL / 2; o > 0; o >>= 1) {
#pragma unroll
    for (int i = 0; i < ND; ++i) D[i] += gxor(gm, D[i], o);
#pragma unroll
    for (int i = 0; i < N; ++i) ev[i] += gxor(gm, ev[i], o);
  }
  const S rr = from_f64<S>(T.crr);
#pragma unroll
  for (int t = 0; t < N; ++t) {
    if (t >= nrow) {
      D[p12(t, t)] = S(1);  // padding row: unit pivot, zero multiplier
      continue;
    }
    const int k = t < cs[0] ? ks[0] : ks[1];
    const int rl = t < cs[0] ? t : t - cs[0];
    ev[t] += rr * from_f64<S>(T.c[(size_t)rl * K + k]);
  }
  // Cholesky of D (every lane), reciprocal diagonal
  bool okd = true;
#pragma unroll
  for (int c = 0; c < N; ++c) {
    S sum = D[p12(c, c)];
#pragma unroll
    for (int k = 0; k < c; ++k) sum -= D[p12(c, k)] * D[p12(c, k)];
    if (!(sum > S(0))) {
      okd = false;
      sum = S(1);
    }
    const S id = rsq(sum);
    D[p12(c, c)] = id;
#pragma unroll
    for (int r = c + 1; r < N; ++r) {
      S t = D[p12(r, c)];
#pragma unroll
      for (int k = 0; k < c; ++k) t -= D[p12(r, k)] * D[p12(c, k)];
      D[p12(r, c)] = t * id;
    }
  }
  if (!okd && l == 0) set_status(status, ST_NOT_SPD);
  if constexpr (ROOT) {
    const int nr = T.nroots;
    if (act) {
      T.y[(size_t)l * M + j] = y;
#pragma unroll
      for (int r = 0; r < RMAX; ++r) T.rX[(size_t)(RMAX * l + r) * nr + rid] = b[1 + r];
    }
#pragma unroll
    for (int i = 0; i < ND; ++i)
      if ((i % GL) == l) T.rLD[(size_t)i * nr + rid] = D[i];
#pragma unroll
    for (int r = 0; r < RMAX; ++r)
      if (l == r) T.re[(size_t)r * nr + rid] = ev[r];
  } else {
    if (act) {
      T.y[(size_t)l * M + j] = y;
#pragma unroll
      for (int t = 0; t < NJ; ++t) T.X[(size_t)(NJ * l + t) * M + j] = b[1 + t];
    }
#pragma unroll
    for (int i = 0; i < ND; ++i)
      if (l == i) T.LD[(size_t)i * M + j] = D[i];
#pragma unroll
    for (int r = 0; r < NJ; ++r)
      if (l == r) T.e[(size_t)r * M + j] = ev[r];
    // contribution to the parent (its rest frame): U = Pbar^T L_D^{-T}, v = U L_D^{-1} e
    const int par = T.parent[j];
    S Rp[3], wp[NJ];
    rot_col(B, par, l, Rp);
    lane_rows(J, ks[0], 1 - T.pside[j], Rp, l, wp);
    S wl[N], z[N];
    S vv = S(0);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      S s = ev[i], u = wp[i];
#pragma unroll
      for (int k = 0; k < i; ++k) {
        s -= D[p12(i, k)] * wl[k];
        u -= D[p12(i, k)] * z[k];
      }
      wl[i] = s * D[p12(i, i)];
      z[i] = u * D[p12(i, i)];
      vv += z[i] * wl[i];
    }
    if (act) {
#pragma unroll
      for (int i = 0; i < N; ++i) T.U[(size_t)(NJ * l + i) * M + j] = z[i];
      T.v[(size_t)l * M + j] = vv;
    }
  }
}

// the root of a tree (level 0): its one-sided joints, padded to RMAX rows
template <typename S>
__device__ __forceinline__ void up_root(const DevBodies &B, const DevJoints &J, const DevTreeT<S> &T, int j,
                                        const StepParams &p, int *status, int l, unsigned gm, S *sc) {
  up_body<S, RMAX, true>(B, J, T, j, p, status, l, gm, sc);
}

template <typename S>
__device__ __forceinline__ void up_inner(const DevBodies &B, const DevJoints &J, const DevTreeT<S> &T, int j,
                                         const StepParams &p, int *status, int l, unsigned gm, S *sc) {
  up_body<S, NJ, false>(B, J, T, j, p, status, l, gm, sc);
}

// downward pass of body j: lambda of its parent joint (or of a root's
// one-sided joints), dq, and the state update.  FULL (FP64 form, set when
// J.qf holds the full gradient's frame terms): its own instantiation, so
// that the frozen-frame kernels keep their registers
template <typename S, bool FULL = false>
__device__ __noinline__ void down_one(const DevBodies &B, const DevJoints &J, const DevTreeT<S> &T, int j,
                                      const StepParams &p) {
  const int M = B.M, K = J.K;
  const int par = T.parent[j];
  S dqb[12];
#pragma unroll
  for (int a = 0; a < 12; ++a) dqb[a] = T.y[(size_t)a * M + j];
  if (par >= 0) {
    const int k = T.pjoint[j];
    const int type = J.type[k];
    const int C = type == 0 ? 3 : 5;
    const int pside = 1 - T.pside[j];
    // P dq_parent: rows s_p d_r^T J(p_r) dq_p in the world frame
    S dqp[12];
#pragma unroll
    for (int a = 0; a < 12; ++a) dqp[a] = T.dq[(size_t)a * M + par];
    S pts[2][3], x[2][3], RH[9];
    // every joint's second point and frame are loaded (valid storage for a
    // ball joint too) alongside its type, then a ball joint takes the
    // identity frame: no load waits for the type
    load3(JP<S>::p1(J, pside), K, k, pts[0]);
    load3(JP<S>::p2(J, pside), K, k, pts[1]);
    load_R(JP<S>::RH(J), K, k, RH);
    if (type == 0) {
#pragma unroll
      for (int a = 0; a < 3; ++a) pts[1][a] = S(0);
#pragma unroll
      for (int a = 0; a < 9; ++a) RH[a] = (a % 4 == 0) ? S(1) : S(0);
    }
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int a = 0; a < 3; ++a)
        x[q][a] = dqp[a] * pts[q][0] + dqp[3 + a] * pts[q][1] + dqp[6 + a] * pts[q][2] + dqp[9 + a];
    const S sp = pside == 0 ? S(1) : -S(1);
    // MABD_JACOBIAN_FULL (FP64 form only): when the parent is the joint's
    // body a, its rows also carry the frame term qh_r . axial(X - X^T), X
    // the 3x3 block of the parent's rest-frame displacement R_p^T dq_p
    // MABD_JACOBIAN_FULL: when the parent is the joint's body a, its rows
    // also carry the frame term qh_r . axial(X - X^T), X the 3x3 block of the
    // parent's rest-frame displacement R_p^T dq_p
    S ext[NJ];
#pragma unroll
    for (int r = 0; r < NJ; ++r) ext[r] = S(0);
    if constexpr (FULL && sizeof(S) == 8) {
      if (pside == 0 && type == 1) {
        double Rp[9], xr[12], w[3];
        load_R(B.R, M, par, Rp);
#pragma unroll
        for (int c = 0; c < 3; ++c) mtv3(Rp, dqp + 3 * c, xr + 3 * c);
        xr[9] = xr[10] = xr[11] = 0.0;
        skew_axial(xr, w);
#pragma unroll
        for (int r = 0; r < NJ; ++r) {
          double qh[3];
          load_qf(J.qf, K, k, r, qh);
          ext[r] = qh[0] * w[0] + qh[1] * w[1] + qh[2] * w[2];
        }
      }
    }
    S t[NJ], lam[NJ], LD[15];
#pragma unroll
    for (int i = 0; i < 15; ++i) LD[i] = T.LD[(size_t)i * M + j];
    // rows: R_H's rows 0-2 at the first point, rows 0 and 2 at the second
    // (identity rows for a ball joint, whose rows 3 and 4 are padding)
#pragma unroll
    for (int r = 0; r < NJ; ++r) {
      const int rr = r < 3 ? r : (r == 3 ? 0 : 2);
      const int q = r < 3 ? 0 : 1;
      const S dx = RH[3 * rr] * x[q][0] + RH[3 * rr + 1] * x[q][1] + RH[3 * rr + 2] * x[q][2];
      const S rhs = r < C ? T.e[(size_t)r * M + j] + sp * dx + ext[r] : S(0);
      S s = rhs;
#pragma unroll
      for (int i = 0; i < r; ++i) s -= LD[p12(r, i)] * t[i];
      t[r] = s * LD[p12(r, r)];
    }
#pragma unroll
    for (int i = NJ - 1; i >= 0; --i) {
      S s = t[i];
#pragma unroll
      for (int q = i + 1; q < NJ; ++q) s -= LD[p12(q, i)] * lam[q];
      lam[i] = s * LD[p12(i, i)];
    }
#pragma unroll
    for (int r = 0; r < NJ; ++r)
      if (r < C) put_lambda(T, (size_t)r * K + k, lam[r]);
#pragma unroll
    for (int a = 0; a < 12; ++a)
#pragma unroll
      for (int r = 0; r < NJ; ++r) dqb[a] -= T.X[(size_t)(NJ * a + r) * M + j] * lam[r];
  } else {
    const int rid = T.root_id[j];
    const int nr = T.nroots;
    int n = 0, cs[2] = {0, 0}, ks[2] = {-1, -1};
    for (int w = 0; w < 2; ++w) {
      ks[w] = rid >= 0 ? T.root_joint[(size_t)w * nr + rid] : -1;
      cs[w] = ks[w] < 0 ? 0 : (J.type[ks[w]] == 0 ? 3 : 5);
      n += cs[w];
    }
    // the factor's leading n x n block is the root's own (padding after it)
    S lam[RMAX], t[RMAX];
#pragma unroll 1
    for (int i = 0; i < n; ++i) {
      S s = T.re[(size_t)i * nr + rid];
      for (int q = 0; q < i; ++q) s -= T.rLD[(size_t)p12(i, q) * nr + rid] * t[q];
      t[i] = s * T.rLD[(size_t)p12(i, i) * nr + rid];
    }
#pragma unroll 1
    for (int i = n - 1; i >= 0; --i) {
      S s = t[i];
      for (int q = i + 1; q < n; ++q) s -= T.rLD[(size_t)p12(q, i) * nr + rid] * lam[q];
      lam[i] = s * T.rLD[(size_t)p12(i, i) * nr + rid];
    }
#pragma unroll 1
    for (int r = 0; r < n; ++r) {
      const int w = r < cs[0] ? 0 : 1;
      put_lambda(T, (size_t)(r - (w ? cs[0] : 0)) * K + ks[w], lam[r]);
#pragma unroll
      for (int a = 0; a < 12; ++a) dqb[a] -= T.rX[(size_t)(RMAX * a + r) * nr + rid] * lam[r];
    }
  }
  S R[9];
  load_R(TB<S>::R(B), M, j, R);
#pragma unroll
  for (int blk = 0; blk < 4; ++blk) {
    S dq[3];
    mv3(R, dqb + 3 * blk, dq);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const size_t o = (size_t)(3 * blk + a) * M + j;
      T.dq[o] = dq[a];
      if (!T.dqb) {  // FP64 form: the state update
        B.q[o] += to_f64(dq[a]);
        B.qd[o] = to_f64(dq[a]) * p.inv_h;
      }
    }
  }
  if (T.dqb) {  // mixed form: the rest-frame increment, set or accumulated over the sweeps
#pragma unroll
    for (int a = 0; a < 12; ++a) {
      const size_t o = (size_t)a * M + j;
      const double v = to_f64(dqb[a]);
      T.dqb[o] = T.dqb_add ? T.dqb[o] + v : v;
    }
  }
}

constexpr int GB = 128;       // threads per block of the level kernels
constexpr int GNG = GB / GL;  // lane groups per block

// one level of the upward pass: a lane group per body of order[lo, hi)
template <typename S>
__global__ void __launch_bounds__(GB) k_tree_up_level(DevBodies B, DevJoints J, DevTreeT<S> T, int lo, int hi,
                                                      StepParams p, int *status) {
  __shared__ S scr[GNG][GSC];
  const int g = threadIdx.x / GL, l = threadIdx.x % GL;
  const unsigned gm = 0xFFFFu << (threadIdx.x & 16);
  const int i = lo + blockIdx.x * GNG + g;
  if (i >= hi) return;  // uniform in the group
  const int j = T.order[i];
  if (!MABD_INDEX_OK(j, B.M, status)) return;
  if (T.parent[j] < 0) return;
  if (!MABD_INDEX_OK(T.parent[j], B.M, status) || !MABD_INDEX_OK(T.pjoint[j], J.K, status)) return;
  if (T.ccount[j] > 0 && !(MABD_INDEX_OK(T.cfirst[j], B.M, status) &&
                           MABD_INDEX_OK(T.cfirst[j] + T.ccount[j] - 1, B.M, status)))
    return;
  up_inner<S>(B, J, T, j, p, status, l, gm, scr[g]);
}

// the roots (level 0, bodies lo .. hi - 1), a lane group per root
template <typename S>
__global__ void __launch_bounds__(GB) k_tree_up_root(DevBodies B, DevJoints J, DevTreeT<S> T, int lo, int hi,
                                                     StepParams p, int *status) {
  __shared__ S scr[GNG][GSC];
  const int g = threadIdx.x / GL, l = threadIdx.x % GL;
  const unsigned gm = 0xFFFFu << (threadIdx.x & 16);
  const int j = lo + blockIdx.x * GNG + g;
  if (j >= hi || T.parent[j] >= 0) return;  // uniform in the group
  up_root<S>(B, J, T, j, p, status, l, gm, scr[g]);
}

template <typename S, bool FULL>
__global__ void __launch_bounds__(128) k_tree_down(DevBodies B, DevJoints J, DevTreeT<S> T, int lo, int hi,
                                                   StepParams p) {
  const int j = lo + blockIdx.x * blockDim.x + threadIdx.x;
  if (j < hi) down_one<S, FULL>(B, J, T, j, p);
}

// Consecutive narrow levels [la, lb) of the downward pass in one block of RB
// threads, root first, a block barrier between levels.  A narrow level's
// own launch costs more than its bodies (one thread each: a few loads and a
// 5x5 solve), so a run of them shares one launch.  (The upward pass keeps
// a launch per level: there a body's latency, not the launch, sets the cost.)
constexpr int RB = 256;

template <typename S, bool FULL>
__global__ void __launch_bounds__(RB) k_tree_down_run(DevBodies B, DevJoints J, DevTreeT<S> T, int la, int lb,
                                                      StepParams p) {
  for (int d = la; d < lb; ++d) {
    const int lo = T.lv_lo[d], hi = T.lv_lo[d + 1];
    for (int j = lo + threadIdx.x; j < hi; j += RB) down_one<S, FULL>(B, J, T, j, p);
    __syncthreads();
  }
}

// Persistent kernel, one block of NT threads per tree in the forest's record
// order (deepest trees first): per level of the upward pass the NT / GL lane
// groups take its bodies, then the root, then the downward pass a thread per
// body; a block barrier between levels.
template <typename S, int NT>
__global__ void __launch_bounds__(NT) k_tree_forest(DevBodies B, DevJoints J, DevTreeT<S> T, DevForest F,
                                                    StepParams p, int *status) {
  constexpr int NG = NT / GL;
  __shared__ S scr[NG][GSC];
  const int g = threadIdx.x / GL, l = threadIdx.x % GL;
  const unsigned gm = 0xFFFFu << (threadIdx.x & 16);
  for (int t = blockIdx.x; t < F.ntrees; t += gridDim.x) {
    const int r0 = F.tlvl[t], nl = F.tnl[t];
    for (int d = nl - 1; d >= 1; --d) {
      const int lo = F.lo[r0 + d], hi = F.lo[r0 + d + 1];
      for (int i = lo + g; i < hi; i += NG) up_inner<S>(B, J, T, F.order[i], p, status, l, gm, scr[g]);
      __syncthreads();
    }
    if (g == 0) up_root<S>(B, J, T, F.order[F.lo[r0]], p, status, l, gm, scr[0]);
    __syncthreads();
    for (int d = 0; d < nl; ++d) {
      const int lo = F.lo[r0 + d], hi = F.lo[r0 + d + 1];
      for (int i = lo + threadIdx.x; i < hi; i += NT) {
        if constexpr (sizeof(S) == 8) {
          if (J.qf) down_one<S, true>(B, J, T, F.order[i], p);
          else down_one<S, false>(B, J, T, F.order[i], p);
        } else {
          down_one<S, false>(B, J, T, F.order[i], p);
        }
      }
      __syncthreads();
    }
  }
}

template <typename S>
void launch_tree_forest(const DevBodies &B, const DevJoints &J, const DevTreeT<S> &T, const DevForest &F,
                        const StepParams &p, int *status, cudaStream_t s, int threads) {
  if (F.ntrees <= 0) return;
  if (threads == 32) k_tree_forest<S, 32><<<F.ntrees, 32, 0, s>>>(B, J, T, F, p, status);
  else if (threads == 64) k_tree_forest<S, 64><<<F.ntrees, 64, 0, s>>>(B, J, T, F, p, status);
  else k_tree_forest<S, 128><<<F.ntrees, 128, 0, s>>>(B, J, T, F, p, status);
}

template <typename S>
void launch_tree_up(const DevBodies &B, const DevJoints &J, const DevTreeT<S> &T, int lo, int hi, bool roots,
                    const StepParams &p, int *status, cudaStream_t s) {
  if (hi <= lo) return;
  if (roots) k_tree_up_root<S><<<(hi - lo + GNG - 1) / GNG, GB, 0, s>>>(B, J, T, lo, hi, p, status);
  else k_tree_up_level<S><<<(hi - lo + GNG - 1) / GNG, GB, 0, s>>>(B, J, T, lo, hi, p, status);
}

template <typename S>
void launch_tree_down(const DevBodies &B, const DevJoints &J, const DevTreeT<S> &T, int lo, int hi,
                      const StepParams &p, int * /*status*/, cudaStream_t s) {
  const int n = hi - lo;
  if (n <= 0) return;
  if (sizeof(S) == 8 && J.qf) k_tree_down<S, true><<<(n + 127) / 128, 128, 0, s>>>(B, J, T, lo, hi, p);
  else k_tree_down<S, false><<<(n + 127) / 128, 128, 0, s>>>(B, J, T, lo, hi, p);
}

template <typename S>
void launch_tree_down_run(const DevBodies &B, const DevJoints &J, const DevTreeT<S> &T, int la, int lb,
                          const StepParams &p, cudaStream_t s) {
  if (lb <= la) return;
  if (sizeof(S) == 8 && J.qf) k_tree_down_run<S, true><<<1, RB, 0, s>>>(B, J, T, la, lb, p);
  else k_tree_down_run<S, false><<<1, RB, 0, s>>>(B, J, T, la, lb, p);
}

#define MABD_TREE_INSTANTIATE(S)                                                                   \
  template void launch_tree_down_run<S>(const DevBodies &, const DevJoints &, const DevTreeT<S> &,  \
                                        int, int, const StepParams &, cudaStream_t);               \
  template void launch_tree_forest<S>(const DevBodies &, const DevJoints &, const DevTreeT<S> &,    \
                                      const DevForest &, const StepParams &, int *, cudaStream_t,  \
                                      int);                                                        \
  template void launch_tree_up<S>(const DevBodies &, const DevJoints &, const DevTreeT<S> &, int,   \
                                  int, bool, const StepParams &, int *, cudaStream_t);             \
  template void launch_tree_down<S>(const DevBodies &, const DevJoints &, const DevTreeT<S> &, int, \
                                    int, const StepParams &, int *, cudaStream_t);
MABD_TREE_INSTANTIATE(double)
MABD_TREE_INSTANTIATE(float)
#undef MABD_TREE_INSTANTIATE

}  // namespace mabd
