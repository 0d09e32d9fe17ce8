// Device math shared by the kernels: 3x3 algebra (row-major), the polar
// rotation, the hinge frame and the structured Hbar^{-1} of a body.
#pragma once
#include <cstdint>

#include "mabd_internal.h"
#include "fconv.h"

namespace mabd {

__device__ __forceinline__ double ldg(const double *p) { return __ldg(p); }
// index of the entry that thread t handles under a processing order (CHUNK_ORDER)
__device__ __forceinline__ int ordered(const int32_t *order, int t) { return order ? __ldg(order + t) : t; }

__device__ __forceinline__ void set_status(int *status, int bits) {
  if (status) atomicOr(status, bits);
}

// Index checks of a MABD_DEBUG build: an index that a kernel read from
// memory (a joint's bodies, a tree link, a graph neighbour) is checked
// against its range before use; a bad one sets ST_BOUNDS in the status word
// and the caller skips the access (never a trap).  Other builds compile the
// checks to true.
__device__ __forceinline__ bool index_in_range(long long i, long long n, int *status) {
  if (i >= 0 && i < n) return true;
  set_status(status, ST_BOUNDS);
  return false;
}
#ifdef MABD_DEBUG
#define MABD_INDEX_OK(i, n, status) ::mabd::index_in_range((i), (n), (status))
#else
#define MABD_INDEX_OK(i, n, status) true
#endif

// A(r,c) = q[3c+r] (Eq. abd_dof: vec stacks the columns of A)
__device__ __forceinline__ void A_from_q(const double q[12], double A[9]) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) A[3 * r + c] = q[3 * c + r];
}

template <typename S>
__device__ __forceinline__ void mv3(const S M[9], const S x[3], S y[3]) {
  y[0] = M[0] * x[0] + M[1] * x[1] + M[2] * x[2];
  y[1] = M[3] * x[0] + M[4] * x[1] + M[5] * x[2];
  y[2] = M[6] * x[0] + M[7] * x[1] + M[8] * x[2];
}

template <typename S>
__device__ __forceinline__ void mtv3(const S M[9], const S x[3], S y[3]) {
  y[0] = M[0] * x[0] + M[3] * x[1] + M[6] * x[2];
  y[1] = M[1] * x[0] + M[4] * x[1] + M[7] * x[2];
  y[2] = M[2] * x[0] + M[5] * x[1] + M[8] * x[2];
}

// x(p) = A p + t for the affine coordinates q (Eq. abd)
__device__ __forceinline__ void point_of(const double q[12], const double p[3], double x[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) x[a] = q[a] * p[0] + q[3 + a] * p[1] + q[6 + a] * p[2] + q[9 + a];
}

// gap x_a(pa) - x_b(pb) of two joint points (Eq. ball), evaluated as
// (A_a pa - A_b pb) + (t_a - t_b) so that far-from-origin assemblies keep it
// at round-off of the body size; qb == nullptr: pb is a world point.
__device__ __forceinline__ void gap_of(const double qa[12], const double pa[3], const double *qb,
                                       const double pb[3], double d[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double la = qa[a] * pa[0] + qa[3 + a] * pa[1] + qa[6 + a] * pa[2];
    if (qb) {
      const double lb = qb[a] * pb[0] + qb[3 + a] * pb[1] + qb[6 + a] * pb[2];
      d[a] = (la - lb) + (qa[9 + a] - qb[9 + a]);
    } else {
      d[a] = la + (qa[9 + a] - pb[a]);
    }
  }
}

// Eq. polar: R = A (A^T A)^{-1/2} by Newton's iteration X <- (X + X^{-T})/2,
// X^{-T} = cof(X)/det(X).  Returns a ST_* code (0 on success).
// The first step's determinant is det A, so the step loop also makes the
// det A <= 0 check.  The stopping test compares the squared step with
// 1e-18 |R|^2 = 3e-18 (the iterate tends to a rotation, |R|_F^2 = 3).
__device__ __forceinline__ int polar3(const double A[9], double R[9], int *iters = nullptr) {
  double X[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) X[i] = A[i];
  int it = 0;
  for (; it < 40; ++it) {
    double C[9];
    C[0] = X[4] * X[8] - X[5] * X[7];
    C[1] = X[5] * X[6] - X[3] * X[8];
    C[2] = X[3] * X[7] - X[4] * X[6];
    C[3] = X[2] * X[7] - X[1] * X[8];
    C[4] = X[0] * X[8] - X[2] * X[6];
    C[5] = X[1] * X[6] - X[0] * X[7];
    C[6] = X[1] * X[5] - X[2] * X[4];
    C[7] = X[2] * X[3] - X[0] * X[5];
    C[8] = X[0] * X[4] - X[1] * X[3];
    double d = X[0] * C[0] + X[1] * C[1] + X[2] * C[2];
    if (!(d > 0.0)) return isfinite(d) ? ST_INVERTED : ST_NONFINITE;
    double hid = 0.5 / d;
    double diff = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      double y = 0.5 * X[i] + hid * C[i];
      double dx = y - X[i];
      diff += dx * dx;
      X[i] = y;
    }
    // quadratic convergence: a relative change below 1e-9 leaves an error
    // of order 1e-18 in the iterate just formed
    if (diff <= 3e-18) break;
  }
  if (it == 40) return ST_POLAR_NOCONV;
#pragma unroll
  for (int i = 0; i < 9; ++i) R[i] = X[i];
  if (iters) *iters = it + 1;
  return 0;
}

// *c += v summed over the converged lanes of the warp (one atomic per warp)
__device__ __forceinline__ void count_add(unsigned long long *c, unsigned v) {
  const unsigned mask = __activemask();
  const unsigned sum = __reduce_add_sync(mask, v);
  if ((int)(threadIdx.x & 31) == __ffs(mask) - 1) atomicAdd(c, (unsigned long long)sum);
}

// Sec. 4.3: R_H = I + [v]x + [v]x^2 / (1 + a_y), v = a x e_y = (-a_z, 0, a_x)
__device__ __forceinline__ void hinge_frame(const double a[3], double RH[9]) {
  const double vx = -a[2], vz = a[0];
  const double k = 1.0 / (1.0 + a[1]);
  // [v]x with v = (vx, 0, vz): [[0, -vz, 0], [vz, 0, -vx], [0, vx, 0]]
  // [v]x^2 = v v^T - |v|^2 I
  const double n2 = vx * vx + vz * vz;
  RH[0] = 1.0 + k * (vx * vx - n2);
  RH[1] = -vz;
  RH[2] = k * (vx * vz);
  RH[3] = vz;
  RH[4] = 1.0 - k * n2;
  RH[5] = -vx;
  RH[6] = k * (vz * vx);
  RH[7] = vx;
  RH[8] = 1.0 + k * (vz * vz - n2);
}

// world direction of constraint row r (Eq. ball: identity rows; Eq. hinge:
// rows 0-2 are the rows of R_H, rows 3 and 4 its x and z rows at the second
// point; Eq. prismatic: the x and z rows of R_P at the anchors, x and z at
// the on-axis points, z at the off-axis points)
template <typename S>
__device__ __forceinline__ void row_dir(int type, const S RH[9], int r, S d[3]) {
  if (type == 0) {
    d[0] = r == 0 ? S(1) : S(0);
    d[1] = r == 1 ? S(1) : S(0);
    d[2] = r == 2 ? S(1) : S(0);
  } else {
    // hinge: rows 3, 4 are R_H's x and z rows; universal (R_U in RH): row 3
    // is its a1 row; prismatic (R_P in RH): rows x, z, x, z, z
    const int rr = type == 3 ? ((r == 0 || r == 2) ? 0 : 2) : (r < 3 ? r : (type == 2 ? 1 : (r == 3 ? 0 : 2)));
    // selects, not RH[3 * rr]: a run-time index would put RH in local memory
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = rr == 0 ? RH[a] : (rr == 1 ? RH[3 + a] : RH[6 + a]);
  }
}

__device__ __forceinline__ void load_hinv(const DevBodies &B, int j, double h[16]) {
#pragma unroll
  for (int i = 0; i < 16; ++i) h[i] = ldg(B.hinv + (size_t)i * B.M + j);
}

template <typename S>
__device__ __forceinline__ void load_R(const S *R, int N, int j, S out[9]) {
#pragma unroll
  for (int i = 0; i < 9; ++i) out[i] = R[(size_t)i * N + j];
}

template <typename S>
__device__ __forceinline__ void load12(const S *p, int N, int j, S out[12]) {
#pragma unroll
  for (int i = 0; i < 12; ++i) out[i] = p[(size_t)i * N + j];
}

template <typename S>
__device__ __forceinline__ void load3(const S *p, int N, int j, S out[3]) {
  out[0] = __ldg(p + j);
  out[1] = __ldg(p + (size_t)N + j);
  out[2] = __ldg(p + 2 * (size_t)N + j);
}

// joint points and hinge frames in the precision of the products (the FP32
// copies exist in the mixed-precision forms)
template <typename S> struct JP;
template <> struct JP<double> {
  __device__ static const double *p1(const DevJoints &J, int side) { return side == 0 ? J.pa1 : J.pb1; }
  __device__ static const double *p2(const DevJoints &J, int side) { return side == 0 ? J.pa2 : J.pb2; }
  __device__ static const double *p3(const DevJoints &J, int side) { return side == 0 ? J.pa3 : J.pb3; }
  __device__ static const double *RH(const DevJoints &J) { return J.RH; }
};
template <> struct JP<float> {
  __device__ static const float *p1(const DevJoints &J, int side) { return side == 0 ? J.pa1f : J.pb1f; }
  __device__ static const float *p2(const DevJoints &J, int side) { return side == 0 ? J.pa2f : J.pb2f; }
  __device__ static const float *p3(const DevJoints &J, int side) { return side == 0 ? J.pa3f : J.pb3f; }
  __device__ static const float *RH(const DevJoints &J) { return J.RHf; }
};

__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }

// Rows of joint k on the body with rotation R that is its side `side`
// (0: body a, 1: body b): row r is s [p; w] (x) (R^T d_r) in that body's rest
// frame (frozen frame, Eq. pcpq), s = +1 on a and -1 on b, p the row's point
// and w its translation weight (0 for a point difference).  Writes the
// directions E[r], the points P[0..NP-1], their weights and the point index
// pt[r]; returns C.  NP = 3 holds the prismatic joint's third point pair
// (universal and prismatic joints need it); the solvers and scenes with
// only ball and hinge joints pass NP = 2.
template <typename S, int NP>
__device__ __forceinline__ int joint_rows_rest(const DevJoints &J, int k, int side, const S R[9],
                                               S E[5][3], S (&P)[NP][3], int pt[5], S (&wgt)[NP]) {
  const int K = J.K;
  const int type = J.type[k];
  const S sgn = side == 0 ? S(1) : S(-1);
  load3(JP<S>::p1(J, side), K, k, P[0]);
#pragma unroll
  for (int i = 0; i < NP; ++i) wgt[i] = S(1);
  S RH[9];
  if (type != 0) {
    load3(JP<S>::p2(J, side), K, k, P[1]);
#pragma unroll
    for (int i = 0; i < 9; ++i) RH[i] = JP<S>::RH(J)[(size_t)i * K + k];
  }
  if (NP > 2) {
    if (type == 3) {
      load3(JP<S>::p3(J, side), K, k, P[NP > 2 ? 2 : 0]);
    } else {
#pragma unroll
      for (int a = 0; a < 3; ++a) P[NP > 2 ? 2 : 0][a] = S(0);
    }
  }
  const int C = joint_nrows(type);
  // unrolled over the five possible rows, so that E and pt stay in registers
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    if (r >= C) break;
    S d[3], e[3];
    // two point slots: only ball and hinge joints reach here
    row_dir(NP > 2 ? type : (type == 0 ? 0 : 1), RH, r, d);
    mtv3(R, d, e);
    // the universal joint's row 3: + a1 (x) [l a2; 0] on beta (a point
    // difference: weight 0 on the translation), nothing on alpha
    const S s = (NP > 2 && type == 2 && r == 3) ? (side == 0 ? S(0) : S(1)) : sgn;
    E[r][0] = s * e[0];
    E[r][1] = s * e[1];
    E[r][2] = s * e[2];
    pt[r] = (NP > 2 && type == 3) ? (r >> 1) : (r < 3 ? 0 : 1);
  }
  if (NP > 2 && type == 2) wgt[1] = S(0);
  return C;
}

template <typename S, int NP>
__device__ __forceinline__ int joint_rows_rest(const DevJoints &J, int k, int side, const S R[9],
                                               S E[5][3], S (&P)[NP][3], int pt[5]) {
  S wgt[NP];
  return joint_rows_rest(J, k, side, R, E, P, pt, wgt);
}

// The rows with each row's own point PR[r] and translation weight WR[r]
// (every joint type, three point slots).  The point of a row is picked with
// selects on registers: indexing a 3-point array with a run-time row index
// would put the array in local memory.
// XJ: the scene may hold prismatic joints (three point slots); without, two.
template <typename S, bool XJ = true>
__device__ __forceinline__ int joint_rows_pt(const DevJoints &J, int k, int side, const S R[9], S E[5][3],
                                             S PR[5][3], S WR[5]) {
  constexpr int NP = XJ ? 3 : 2;
  S P[NP][3], wt[NP];
  int pt[5] = {0, 0, 0, 0, 0};
  const int C = joint_rows_rest<S, NP>(J, k, side, R, E, P, pt, wt);
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const int q = pt[r];
#pragma unroll
    for (int a = 0; a < 3; ++a) PR[r][a] = q == 0 ? P[0][a] : (q == 1 || NP == 2 ? P[1][a] : P[NP - 1][a]);
    WR[r] = q == 0 ? wt[0] : (q == 1 || NP == 2 ? wt[1] : wt[NP - 1]);
  }
  return C;
}

// Sec. 4.5 prismatic joint frame R_P = [x~; y~; z~] (rows), frozen at q_n and
// attached to alpha (Sec. 5.1 writes a joint frame as a constant rotation
// times alpha's R^T): y~ = Ra ua (the sliding axis), x~ = Ra ca made normal
// to y~ (ca: alpha's reference direction, any length), z~ = x~ x y~
template <typename S>
__device__ __forceinline__ void prismatic_frame(const S Ra[9], const S ua[3], const S ca[3], S RP[9]) {
  S y[3], x[3];
  mv3(Ra, ua, y);
  mv3(Ra, ca, x);
  S n = rsq(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
  y[0] *= n; y[1] *= n; y[2] *= n;
  const S d = y[0] * x[0] + y[1] * x[1] + y[2] * x[2];
  x[0] -= d * y[0]; x[1] -= d * y[1]; x[2] -= d * y[2];
  n = rsq(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  x[0] *= n; x[1] *= n; x[2] *= n;
  RP[0] = x[0]; RP[1] = x[1]; RP[2] = x[2];
  RP[3] = y[0]; RP[4] = y[1]; RP[5] = y[2];
  RP[6] = x[1] * y[2] - x[2] * y[1];
  RP[7] = x[2] * y[0] - x[0] * y[2];
  RP[8] = x[0] * y[1] - x[1] * y[0];
}

// Sec. 4.4 universal joint frame R_U = [a1 x a2; a1; a2] (rows), frozen at
// q_n: a1 = Ra ua (alpha's axis), a2 = Rb vb (beta's axis) made normal to a1
// (Gram-Schmidt), both normalised
template <typename S>
__device__ __forceinline__ void universal_frame(const S Ra[9], const S ua[3], const S Rb[9], const S vb[3],
                                                S RU[9]) {
  S a1[3], w[3];
  mv3(Ra, ua, a1);
  mv3(Rb, vb, w);
  S n = rsq(a1[0] * a1[0] + a1[1] * a1[1] + a1[2] * a1[2]);
  a1[0] *= n; a1[1] *= n; a1[2] *= n;
  const S d = a1[0] * w[0] + a1[1] * w[1] + a1[2] * w[2];
  w[0] -= d * a1[0]; w[1] -= d * a1[1]; w[2] -= d * a1[2];
  n = rsq(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
  w[0] *= n; w[1] *= n; w[2] *= n;
  RU[0] = a1[1] * w[2] - a1[2] * w[1];
  RU[1] = a1[2] * w[0] - a1[0] * w[2];
  RU[2] = a1[0] * w[1] - a1[1] * w[0];
  RU[3] = a1[0]; RU[4] = a1[1]; RU[5] = a1[2];
  RU[6] = w[0]; RU[7] = w[1]; RU[8] = w[2];
}

// w = [p; wt] (x) e as a 12-vector (wt = 0: a point difference, no
// translation part)
template <typename S>
__device__ __forceinline__ void kron_row_w(const S p[3], S wt, const S e[3], S w[12]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    w[a] = p[0] * e[a];
    w[3 + a] = p[1] * e[a];
    w[6 + a] = p[2] * e[a];
    w[9 + a] = wt * e[a];
  }
}

template <typename S>
__device__ __forceinline__ void kron_row(const S p[3], const S e[3], S w[12]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    w[a] = p[0] * e[a];
    w[3 + a] = p[1] * e[a];
    w[6 + a] = p[2] * e[a];
    w[9 + a] = e[a];
  }
}

// y = Hbar^{-1} v with the structured inverse h[16] (see mabd_internal.h)
template <typename S>
__device__ __forceinline__ void hinv_apply(const S h[16], const S v[12], S y[12]) {
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

// Mbar(p, q) = ([p;1] (x) I)^T Hbar^{-1} ([q;1] (x) I), the 3x3 compliance between
// two rest-frame points of a body, from the structured inverse h[16]: translation h[0]; the 3x3
// block X of A's diagonal entries (h[1..6]); transpose pairs
// (A(1,0), A(0,1)) h[7..9], (A(2,0), A(0,2)) h[10..12], (A(2,1), A(1,2)) h[13..15].
template <typename T>
__device__ __forceinline__ void mbar(const T h[16], const T p[3], const T q[3], T Mb[3][3]) {
  const T p0q0 = p[0] * q[0], p1q1 = p[1] * q[1], p2q2 = p[2] * q[2];
  Mb[0][0] = h[0] + h[1] * p0q0 + h[9] * p1q1 + h[12] * p2q2;
  Mb[1][1] = h[0] + h[4] * p1q1 + h[7] * p0q0 + h[15] * p2q2;
  Mb[2][2] = h[0] + h[6] * p2q2 + h[10] * p0q0 + h[13] * p1q1;
  const T p0q1 = p[0] * q[1], p1q0 = p[1] * q[0];
  const T p0q2 = p[0] * q[2], p2q0 = p[2] * q[0];
  const T p1q2 = p[1] * q[2], p2q1 = p[2] * q[1];
  Mb[0][1] = h[2] * p0q1 + h[8] * p1q0;
  Mb[1][0] = h[2] * p1q0 + h[8] * p0q1;
  Mb[0][2] = h[3] * p0q2 + h[11] * p2q0;
  Mb[2][0] = h[3] * p2q0 + h[11] * p0q2;
  Mb[1][2] = h[5] * p1q2 + h[14] * p2q1;
  Mb[2][1] = h[5] * p2q1 + h[14] * p1q2;
}

// out[r][c] (r < NA, c < NB) = Ea[:, ca[r]]^T Mb Eb[:, cb[c]]
template <int NA, int NB, typename T>
__device__ __forceinline__ void project(const T Ea[3][3], const int ca[3], const T Mb[3][3],
                                        const T Eb[3][3], const int cb[3], T out[3][3]) {
  T tmp[3][NB];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < NB; ++c)
      tmp[a][c] = Mb[a][0] * Eb[0][cb[c]] + Mb[a][1] * Eb[1][cb[c]] + Mb[a][2] * Eb[2][cb[c]];
#pragma unroll
  for (int r = 0; r < NA; ++r)
#pragma unroll
    for (int c = 0; c < NB; ++c)
      out[r][c] = Ea[0][ca[r]] * tmp[0][c] + Ea[1][ca[r]] * tmp[1][c] + Ea[2][ca[r]] * tmp[2][c];
}

// atomic max of a non-negative double through its bit pattern
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *addr, double v) {
  if (!(v >= 0.0)) v = __longlong_as_double(0x7ff0000000000000ULL);  // NaN -> +inf
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

// ---- MABD_JACOBIAN_FULL (Sec. 5.1, Eq. constraint_gradient / r_gradient) ----
// The joint frame is attached to body a (R_J = dR R_a^T), so a row n . d
// (world direction n, world gap d of its point pair) also changes through
// R_J: by omega . (n x d), omega = R K axial(R^T dA - dA^T R) the world
// rotation rate of a's polar factor, K = (tr(P) I - P)^{-1}, P = R^T A
// (A = R P gives R^T dA - dA^T R = Omega P + P Omega = [(tr(P) I - P) w]x
// with R^T dR = Omega = [w]x).  In a's rest frame the term acting on a
// 12-vector x is qh . axial(X - X^T), X the 3x3 block of x (x[3c + r] =
// X(r, c)) and qh = K R^T (n x d).

// KRt = K R^T for body a
__device__ __forceinline__ void full_frame_map(const double A[9], const double R[9], double KRt[9]) {
  double P[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) P[3 * r + c] = R[r] * A[c] + R[3 + r] * A[3 + c] + R[6 + r] * A[6 + c];
  const double tr = P[0] + P[4] + P[8];
  // Ms = tr(P) I - sym(P) (symmetric, about 2 I near rigid states)
  const double m00 = tr - P[0], m11 = tr - P[4], m22 = tr - P[8];
  const double m01 = -0.5 * (P[1] + P[3]), m02 = -0.5 * (P[2] + P[6]), m12 = -0.5 * (P[5] + P[7]);
  const double c00 = m11 * m22 - m12 * m12, c01 = m02 * m12 - m01 * m22, c02 = m01 * m12 - m02 * m11;
  const double c11 = m00 * m22 - m02 * m02, c12 = m01 * m02 - m00 * m12, c22 = m00 * m11 - m01 * m01;
  const double inv = 1.0 / (m00 * c00 + m01 * c01 + m02 * c02);
  const double K[9] = {c00 * inv, c01 * inv, c02 * inv, c01 * inv, c11 * inv, c12 * inv,
                       c02 * inv, c12 * inv, c22 * inv};
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) KRt[3 * r + c] = K[3 * r] * R[3 * c] + K[3 * r + 1] * R[3 * c + 1] + K[3 * r + 2] * R[3 * c + 2];
}

// qh = KRt (n x d)
__device__ __forceinline__ void full_row_vec(const double KRt[9], const double n[3], const double d[3],
                                             double qh[3]) {
  const double m[3] = {n[1] * d[2] - n[2] * d[1], n[2] * d[0] - n[0] * d[2], n[0] * d[1] - n[1] * d[0]};
  mv3(KRt, m, qh);
}

// axial(X - X^T) of the 3x3 block of a rest-frame 12-vector
__device__ __forceinline__ void skew_axial(const double x[12], double w[3]) {
  w[0] = x[5] - x[7];
  w[1] = x[6] - x[2];
  w[2] = x[1] - x[3];
}

// g += s * (the transpose of x -> qh . axial(X - X^T)) = s [qh]x on X
__device__ __forceinline__ void add_skew_force(const double qh[3], double s, double g[12]) {
  g[5] += s * qh[0];
  g[7] -= s * qh[0];
  g[6] += s * qh[1];
  g[2] -= s * qh[1];
  g[1] += s * qh[2];
  g[3] -= s * qh[2];
}

__device__ __forceinline__ void load_qf(const double *qf, int K, int k, int r, double qh[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) qh[i] = qf[(size_t)(3 * r + i) * K + k];
}

}  // namespace mabd
