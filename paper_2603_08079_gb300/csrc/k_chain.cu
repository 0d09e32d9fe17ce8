// Chain path of one M-ABD step (FP64), Sec. 5.2:
//   k_chain_gram  per body j: the Gram blocks of its (at most two) joints,
//                 G_kj H_j^{-1} G_k'j^T (Eq. chain-Schur-blocks), formed in the
//                 body's rest frame with the structured Hbar^{-1};
//   k_cr_*        block cyclic reduction of the block-tridiagonal dual
//                 (Eq. chain-btd) with every block padded to 5x5 (a ball's two
//                 extra rows carry an identity diagonal and decouple exactly).
// Packed lower-triangular 5x5 storage: entry (r, c), r >= c, at r(r+1)/2 + c.
#include "mabd_device.cuh"

namespace mabd {

__device__ __forceinline__ int pk(int r, int c) { return r >= c ? r * (r + 1) / 2 + c : c * (c + 1) / 2 + r; }

// ---------------------------------------------------------------------------
// per-body Gram blocks
// ---------------------------------------------------------------------------
// A constraint row of joint k on body j is w = s ([p; 1] (x) d) in world
// coordinates (Eq. ball / hinge, frozen frame), with s = +1 on body a and -1 on
// body b.  In the rest frame it is [p; 1] (x) e with e = s R^T d, and
//   w^T H^{-1} w' = e^T Mbar(p, p') e',  Mbar(p, p') = ([p;1] (x) I)^T Hbar^{-1} ([p';1] (x) I)
// (Eq. abd_final): the 3x3 compliance between two points of the body.  Rows
// are grouped by point (a ball: 3 rows at its anchor; a hinge: 3 rows at the
// anchor and 2 at the second point), so each Gram block is E^T Mbar E' with
// the group's rest-frame directions E.

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

// Gram blocks of body j with products in T (double: the FP64 form; float:
// the mixed form, inputs rounded to FP32); the blocks are stored in FP64.
template <typename T> struct GP;
template <> struct GP<double> {
  __device__ static const double *R(const DevBodies &B) { return B.R; }
  __device__ static const double *RH(const DevJoints &J) { return J.RH; }
  __device__ static const double *p1(const DevJoints &J, int side) { return side == 0 ? J.pa1 : J.pb1; }
  __device__ static const double *p2(const DevJoints &J, int side) { return side == 0 ? J.pa2 : J.pb2; }
};
template <> struct GP<float> {
  __device__ static const float *R(const DevBodies &B) { return B.Rf; }
  __device__ static const float *RH(const DevJoints &J) { return J.RHf; }
  __device__ static const float *p1(const DevJoints &J, int side) { return side == 0 ? J.pa1f : J.pb1f; }
  __device__ static const float *p2(const DevJoints &J, int side) { return side == 0 ? J.pa2f : J.pb2f; }
};

template <typename T, typename HT>
__device__ __forceinline__ void chain_gram_body(const DevBodies &B, const DevJoints &J,
                                                const DevIncidence &I, const DevChain &C,
                                                const HT *hinv, int j) {
  if (B.fixed[j]) return;
  const int e0 = I.off[j];
  const int n = I.off[j + 1] - e0;
  if (n <= 0 || n > 2) return;  // a chain body has one or two joints
  const int M = B.M, K = J.K;
  T R[9], h[16];
#pragma unroll
  for (int i = 0; i < 9; ++i) R[i] = GP<T>::R(B)[(size_t)i * M + j];
#pragma unroll
  for (int i = 0; i < 16; ++i) h[i] = (T)__ldg(hinv + (size_t)i * M + j);
  // per slot: directions E (rest frame, columns = rows' directions), points
  T E[2][3][3], P[2][2][3];
  int kk[2], ty[2];
  for (int s = 0; s < n; ++s) {
    const int k = I.joint[e0 + s];
    const int side = I.side[e0 + s];
    const int type = J.type[k];
    kk[s] = k;
    ty[s] = type;
    const T sgn = side == 0 ? T(1) : T(-1);
    const T *p1 = GP<T>::p1(J, side);
#pragma unroll
    for (int a = 0; a < 3; ++a) P[s][0][a] = __ldg(p1 + (size_t)a * K + k);
    if (type == 1) {
      const T *p2 = GP<T>::p2(J, side);
#pragma unroll
      for (int a = 0; a < 3; ++a) P[s][1][a] = __ldg(p2 + (size_t)a * K + k);
      T RH[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) RH[i] = GP<T>::RH(J)[(size_t)i * K + k];
      // E = s R^T R_H^T: column r is s R^T (row r of R_H)
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int a = 0; a < 3; ++a)
          E[s][a][r] = sgn * (R[a] * RH[3 * r] + R[3 + a] * RH[3 * r + 1] + R[6 + a] * RH[3 * r + 2]);
    } else {
      // E = s R^T
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int r = 0; r < 3; ++r) E[s][a][r] = sgn * R[3 * r + a];
    }
  }
  const int c012[3] = {0, 1, 2}, c02[3] = {0, 2, 0};
  T Mb[3][3], blk[3][3];
  // self blocks of each joint -> its slot (lower body: Dfirst, upper: Dsecond)
  for (int s = 0; s < n; ++s) {
    double *dst = C.islot[e0 + s] == 0 ? C.Dfirst : C.Dsecond;
    const int k = kk[s];
    double Dp[15];
#pragma unroll
    for (int i = 0; i < 15; ++i) Dp[i] = 0.0;
    mbar(h, P[s][0], P[s][0], Mb);
    project<3, 3>(E[s], c012, Mb, E[s], c012, blk);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c <= r; ++c) Dp[pk(r, c)] = (double)blk[r][c];
    if (ty[s] == 1) {
      mbar(h, P[s][1], P[s][0], Mb);                      // rows 3-4 x rows 0-2
      project<2, 3>(E[s], c02, Mb, E[s], c012, blk);
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) Dp[pk(3 + r, c)] = (double)blk[r][c];
      mbar(h, P[s][1], P[s][1], Mb);                      // rows 3-4 x rows 3-4
      project<2, 2>(E[s], c02, Mb, E[s], c02, blk);
      Dp[pk(3, 3)] = (double)blk[0][0];
      Dp[pk(4, 3)] = (double)blk[1][0];
      Dp[pk(4, 4)] = (double)blk[1][1];
    }
#pragma unroll
    for (int i = 0; i < 15; ++i) dst[(size_t)i * K + k] = Dp[i];
  }
  if (n == 2) {
    // coupling of the two joints: rows of joint 0 x rows of joint 1 -> B[k0]
    double Bp[25];
#pragma unroll
    for (int i = 0; i < 25; ++i) Bp[i] = 0.0;
    mbar(h, P[0][0], P[1][0], Mb);
    project<3, 3>(E[0], c012, Mb, E[1], c012, blk);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) Bp[5 * r + c] = (double)blk[r][c];
    if (ty[1] == 1) {
      mbar(h, P[0][0], P[1][1], Mb);
      project<3, 2>(E[0], c012, Mb, E[1], c02, blk);
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) Bp[5 * r + 3 + c] = (double)blk[r][c];
    }
    if (ty[0] == 1) {
      mbar(h, P[0][1], P[1][0], Mb);
      project<2, 3>(E[0], c02, Mb, E[1], c012, blk);
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) Bp[5 * (3 + r) + c] = (double)blk[r][c];
      if (ty[1] == 1) {
        mbar(h, P[0][1], P[1][1], Mb);
        project<2, 2>(E[0], c02, Mb, E[1], c02, blk);
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
          for (int c = 0; c < 2; ++c) Bp[5 * (3 + r) + 3 + c] = (double)blk[r][c];
      }
    }
    const int k0 = kk[0];
#pragma unroll
    for (int i = 0; i < 25; ++i) C.B[(size_t)i * K + k0] = Bp[i];
  }
}

__global__ void __launch_bounds__(128) k_chain_gram(DevBodies B, DevJoints J, DevIncidence I,
                                                    DevChain C) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < B.M) chain_gram_body<double>(B, J, I, C, B.hinv, j);
}

// mixed-precision form: the same blocks with FP32 products
__global__ void __launch_bounds__(128) k_mx_chain_gram(DevBodies B, DevJoints J, DevIncidence I,
                                                       DevChain C) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < B.M) chain_gram_body<float>(B, J, I, C, B.hinvf, j);
}

// ---------------------------------------------------------------------------
// 5x5 helpers (full row-major in registers)
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool chol5(const double A[25], double L[25]) {
  bool ok = true;
#pragma unroll
  for (int i = 0; i < 25; ++i) L[i] = 0.0;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    double s = A[5 * c + c];
#pragma unroll
    for (int k = 0; k < c; ++k) s -= L[5 * c + k] * L[5 * c + k];
    if (!(s > 0.0)) {
      ok = false;
      s = 1.0;
    }
    const double d = sqrt(s);
    const double id = 1.0 / d;
    L[5 * c + c] = d;
#pragma unroll
    for (int r = c + 1; r < 5; ++r) {
      double t = A[5 * r + c];
#pragma unroll
      for (int k = 0; k < c; ++k) t -= L[5 * r + k] * L[5 * c + k];
      L[5 * r + c] = t * id;
    }
  }
  return ok;
}

// x = L^{-1} b
__device__ __forceinline__ void lsolve5(const double L[25], const double b[5], double x[5]) {
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    double s = b[i];
#pragma unroll
    for (int k = 0; k < i; ++k) s -= L[5 * i + k] * x[k];
    x[i] = s / L[5 * i + i];
  }
}

// x = L^{-T} b
__device__ __forceinline__ void ltsolve5(const double L[25], const double b[5], double x[5]) {
#pragma unroll
  for (int i = 4; i >= 0; --i) {
    double s = b[i];
#pragma unroll
    for (int k = i + 1; k < 5; ++k) s -= L[5 * k + i] * x[k];
    x[i] = s / L[5 * i + i];
  }
}

// level loaders (level 0 assembles from the per-body parts; its row n is
// joint n - C.off, and a row before the first joint is a decoupled identity
// row whose multiplier is zero)
__device__ __forceinline__ void ld_D(const DevChain &C, const DevJoints &J, const CRLevel &L,
                                     int level, int n, double D[25]) {
  double p[15];
  if (level == 0) {
    const int k = n - C.off;
    if (k < 0) {
#pragma unroll
      for (int i = 0; i < 15; ++i) p[i] = 0.0;
#pragma unroll
      for (int r = 0; r < 5; ++r) p[pk(r, r)] = 1.0;
    } else {
      const uint8_t f = C.jflags[k];
#pragma unroll
      for (int i = 0; i < 15; ++i) {
        double v = 0.0;
        if (f & 1) v += C.Dfirst[(size_t)i * C.K + k];
        if (f & 2) v += C.Dsecond[(size_t)i * C.K + k];
        p[i] = v;
      }
      if (J.type[k] == 0) {
        p[pk(3, 3)] = 1.0;
        p[pk(4, 4)] = 1.0;
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < 15; ++i) p[i] = L.D[(size_t)i * L.N + n];
  }
#pragma unroll
  for (int r = 0; r < 5; ++r)
#pragma unroll
    for (int c = 0; c < 5; ++c) D[5 * r + c] = p[pk(r, c)];
}

__device__ __forceinline__ void ld_B(const DevChain &C, const CRLevel &L, int level, int n,
                                     double Bm[25]) {
  if (level == 0) {
    const int k = n - C.off;
    const bool has = k >= 0 && (C.jflags[k] & 4);
#pragma unroll
    for (int i = 0; i < 25; ++i) Bm[i] = has ? C.B[(size_t)i * C.K + k] : 0.0;
  } else {
#pragma unroll
    for (int i = 0; i < 25; ++i) Bm[i] = L.B[(size_t)i * L.N + n];
  }
}

__device__ __forceinline__ void ld_b(const DevChain &C, const DevJoints &J, const CRLevel &L,
                                     int level, int n, double b[5]) {
  if (level == 0) {
    const int k = n - C.off;
    const int Cs = k < 0 ? 0 : (J.type[k] == 0 ? 3 : 5);
#pragma unroll
    for (int r = 0; r < 5; ++r) b[r] = r < Cs ? J.b[(size_t)r * J.K + k] : 0.0;
  } else {
#pragma unroll
    for (int r = 0; r < 5; ++r) b[r] = L.b[(size_t)r * L.N + n];
  }
}

// Factor record of an eliminated row (70 doubles): L (packed 15, with the
// reciprocals of its diagonal stored on the diagonal), Ya (25), Yb (25), y (5).
// Contributions to a neighbour: packed 15 + 5.  Blocks keep the 5x5 padded
// layout in memory; the arithmetic runs on the true sizes (3 or 5 rows, and 0
// for a missing right neighbour), chosen per row from the joint types.

// size of row n at `level`: that row is level-0 row n * 2^level, i.e. joint
// n * 2^level - C.off (an identity row of size 3 before the first joint)
__device__ __forceinline__ int row_size(const DevChain &C, const DevJoints &J, int level, int n) {
  const long k = ((long)n << level) - C.off;
  return (k < 0 || J.type[k] == 0) ? 3 : 5;
}

template <int CN, int CL, int CR>
__device__ __forceinline__ void reduce_row(const DevChain &C, const DevJoints &J, const CRLevel &cur,
                                           int level, int n, int m, int Nh, double *cL, double *cR,
                                           double *Bn, int *status, size_t cstride = 0, int cidx = -1,
                                           bool write_fac = true) {
  // contributions go to cL/cR/Bn[(i) * cstride + cidx]; by default the
  // global arrays of the level ([i][Nh], index m)
  if (cstride == 0) {
    cstride = (size_t)Nh;
    cidx = m;
  }
  // D_n, B_{n-1} (CL x CN), B_n (CN x CR), b_n
  double D[25], Bl[25], Br[25], bn[5];
  ld_D(C, J, cur, level, n, D);
  ld_B(C, cur, level, n - 1, Bl);
  if (CR > 0) ld_B(C, cur, level, n, Br);
  ld_b(C, J, cur, level, n, bn);
  // Cholesky with reciprocal diagonal
  double L[CN][CN], id[CN];
  bool ok = true;
#pragma unroll
  for (int c = 0; c < CN; ++c) {
    double sum = D[5 * c + c];
#pragma unroll
    for (int k = 0; k < c; ++k) sum -= L[c][k] * L[c][k];
    if (!(sum > 0.0)) {
      ok = false;
      sum = 1.0;
    }
    id[c] = rsqrt(sum);
    L[c][c] = sum * id[c];
#pragma unroll
    for (int r = c + 1; r < CN; ++r) {
      double t = D[5 * r + c];
#pragma unroll
      for (int k = 0; k < c; ++k) t -= L[r][k] * L[c][k];
      L[r][c] = t * id[c];
    }
  }
  if (!ok) set_status(status, ST_NOT_SPD);
  // Ya = L^{-1} B_{n-1}^T (CN x CL), Yb = L^{-1} B_n (CN x CR), y = L^{-1} b
  double Ya[CN][CL > 0 ? CL : 1], Yb[CN][CR > 0 ? CR : 1], y[CN];
#pragma unroll
  for (int i = 0; i < CN; ++i) {
#pragma unroll
    for (int c = 0; c < CL; ++c) {
      double t = Bl[5 * c + i];
#pragma unroll
      for (int k = 0; k < i; ++k) t -= L[i][k] * Ya[k][c];
      Ya[i][c] = t * id[i];
    }
#pragma unroll
    for (int c = 0; c < CR; ++c) {
      double t = Br[5 * i + c];
#pragma unroll
      for (int k = 0; k < i; ++k) t -= L[i][k] * Yb[k][c];
      Yb[i][c] = t * id[i];
    }
    double t = bn[i];
#pragma unroll
    for (int k = 0; k < i; ++k) t -= L[i][k] * y[k];
    y[i] = t * id[i];
  }
  double *f = cur.fac;
  if (write_fac) {
    int o = 0;
#pragma unroll
    for (int r = 0; r < 5; ++r)
#pragma unroll
      for (int c = 0; c <= r; ++c) {
        double v = 0.0;
        if (r < CN) v = (r == c) ? id[r] : L[r][c];
        f[(size_t)(o++) * Nh + m] = v;
      }
#pragma unroll
    for (int r = 0; r < 5; ++r)
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        f[(size_t)(15 + 5 * r + c) * Nh + m] = (r < CN && c < CL) ? Ya[r][c] : 0.0;
        f[(size_t)(40 + 5 * r + c) * Nh + m] = (r < CN && c < CR) ? Yb[r][c] : 0.0;
      }
#pragma unroll
    for (int r = 0; r < 5; ++r) f[(size_t)(65 + r) * Nh + m] = r < CN ? y[r] : 0.0;
  }
  // neighbour updates: -Ya^T Ya, -Ya^T y to row n-1; -Yb^T Yb, -Yb^T y to row n+1;
  // new coupling -Ya^T Yb between them
#pragma unroll
  for (int r = 0; r < 5; ++r) {
#pragma unroll
    for (int c = 0; c <= r; ++c) {
      double sa = 0.0, sb = 0.0;
      if (r < CL && c < CL) {
#pragma unroll
        for (int t = 0; t < CN; ++t) sa += Ya[t][r] * Ya[t][c];
      }
      if (r < CR && c < CR) {
#pragma unroll
        for (int t = 0; t < CN; ++t) sb += Yb[t][r] * Yb[t][c];
      }
      cL[(size_t)pk(r, c) * cstride + cidx] = sa;
      cR[(size_t)pk(r, c) * cstride + cidx] = sb;
    }
    double ta = 0.0, tb = 0.0;
    if (r < CL) {
#pragma unroll
      for (int t = 0; t < CN; ++t) ta += Ya[t][r] * y[t];
    }
    if (r < CR) {
#pragma unroll
      for (int t = 0; t < CN; ++t) tb += Yb[t][r] * y[t];
    }
    cL[(size_t)(15 + r) * cstride + cidx] = ta;
    cR[(size_t)(15 + r) * cstride + cidx] = tb;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      double sab = 0.0;
      if (r < CL && c < CR) {
#pragma unroll
        for (int t = 0; t < CN; ++t) sab += Ya[t][r] * Yb[t][c];
      }
      Bn[(size_t)(5 * r + c) * cstride + cidx] = -sab;
    }
  }
}

// Odd row n = 2m+1 of the current level:
//   L L^T = D_n, Ya = L^{-1} B_{n-1}^T, Yb = L^{-1} B_n, y = L^{-1} b_n;
//   row n-1 receives -Ya^T Ya, -Ya^T y; row n+1 receives -Yb^T Yb, -Yb^T y;
//   the new coupling between rows n-1 and n+1 is -Ya^T Yb.
__global__ void __launch_bounds__(128) k_cr_reduce(DevChain C, DevJoints J, CRLevel cur, int level,
                                                   double *cL, double *cR, double *Bn, int *status) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = 2 * m + 1;
  const int N = cur.N;
  if (n >= N) return;
  const int Nh = N / 2;
  const int cn = row_size(C, J, level, n), cl = row_size(C, J, level, n - 1);
  const int cr = n + 1 < N ? row_size(C, J, level, n + 1) : 0;
  const int code = (cn == 5 ? 9 : 0) + (cl == 5 ? 3 : 0) + (cr == 5 ? 2 : (cr == 3 ? 1 : 0));
  switch (code) {
#define RED(CODE, A, B, D_) \
  case CODE: reduce_row<A, B, D_>(C, J, cur, level, n, m, Nh, cL, cR, Bn, status); break;
    RED(0, 3, 3, 0) RED(1, 3, 3, 3) RED(2, 3, 3, 5)
    RED(3, 3, 5, 0) RED(4, 3, 5, 3) RED(5, 3, 5, 5)
    RED(9, 5, 3, 0) RED(10, 5, 3, 3) RED(11, 5, 3, 5)
    RED(12, 5, 5, 0) RED(13, 5, 5, 3) RED(14, 5, 5, 5)
#undef RED
    default: break;
  }
}

// Even row e = 2m becomes row m of the next level.
__global__ void __launch_bounds__(128) k_cr_combine(DevChain C, DevJoints J, CRLevel cur, int level,
                                                    CRLevel next, const double *cL,
                                                    const double *cR, const double *Bn) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= next.N) return;
  const int e = 2 * m;
  const int N = cur.N, Nh = N / 2;
  double D[25], b[5];
  ld_D(C, J, cur, level, e, D);
  ld_b(C, J, cur, level, e, b);
  const bool right = e + 1 < N;  // odd row e+1 exists (its index m)
  const bool left = e >= 1;      // odd row e-1 exists (its index m-1)
#pragma unroll
  for (int r = 0; r < 5; ++r)
#pragma unroll
    for (int c = 0; c <= r; ++c) {
      double v = D[5 * r + c];
      if (right) v -= cL[(size_t)pk(r, c) * Nh + m];
      if (left) v -= cR[(size_t)pk(r, c) * Nh + m - 1];
      next.D[(size_t)pk(r, c) * next.N + m] = v;
    }
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    double v = b[r];
    if (right) v -= cL[(size_t)(15 + r) * Nh + m];
    if (left) v -= cR[(size_t)(15 + r) * Nh + m - 1];
    next.b[(size_t)r * next.N + m] = v;
  }
#pragma unroll
  for (int i = 0; i < 25; ++i) next.B[(size_t)i * next.N + m] = right ? Bn[(size_t)i * Nh + m] : 0.0;
}

// One cyclic-reduction level in one launch.  Block b owns the odd rows
// m in [b*(CRF-1), (b+1)*(CRF-1)); its last thread redoes the first odd row
// of the next block as a halo (no factor write).  After the eliminations the
// contributions meet in shared memory and thread t forms next-level row
// m+1 (even row 2m+2) from its own right contribution and the left
// contribution and new coupling of thread t+1; block 0 also forms row 0.
constexpr int CRF = 64;

template <int CN, int CL, int CR>
__device__ __forceinline__ void reduce_row_s(const DevChain &C, const DevJoints &J, const CRLevel &cur,
                                             int level, int n, int m, int Nh, double *sc, int t,
                                             int *status, bool write_fac) {
  reduce_row<CN, CL, CR>(C, J, cur, level, n, m, Nh, sc, sc + 20 * CRF, sc + 40 * CRF, status,
                         (size_t)CRF, t, write_fac);
}

__device__ __forceinline__ void reduce_any(const DevChain &C, const DevJoints &J, const CRLevel &cur,
                                           int level, int n, int m, int Nh, double *sc, int t,
                                           int *status, bool write_fac) {
  const int N = cur.N;
  const int cn = row_size(C, J, level, n), cl = row_size(C, J, level, n - 1);
  const int cr = n + 1 < N ? row_size(C, J, level, n + 1) : 0;
  const int code = (cn == 5 ? 9 : 0) + (cl == 5 ? 3 : 0) + (cr == 5 ? 2 : (cr == 3 ? 1 : 0));
  switch (code) {
#define RED(CODE, A, B_, D_) \
  case CODE: reduce_row_s<A, B_, D_>(C, J, cur, level, n, m, Nh, sc, t, status, write_fac); break;
    RED(0, 3, 3, 0) RED(1, 3, 3, 3) RED(2, 3, 3, 5)
    RED(3, 3, 5, 0) RED(4, 3, 5, 3) RED(5, 3, 5, 5)
    RED(9, 5, 3, 0) RED(10, 5, 3, 3) RED(11, 5, 3, 5)
    RED(12, 5, 5, 0) RED(13, 5, 5, 3) RED(14, 5, 5, 5)
#undef RED
    default: break;
  }
}

// next-level row mm from even row e = 2 mm: D_e - right part of the odd row
// on its left (index mm-1, `sl`) - left part of the odd row on its right
// (index mm, `sr`, which also carries the new coupling)
__device__ __forceinline__ void combine_row(const DevChain &C, const DevJoints &J, const CRLevel &cur,
                                            int level, const CRLevel &next, int mm, const double *sc,
                                            int tl, int tr) {
  const int e = 2 * mm;
  double D[25], b[5];
  ld_D(C, J, cur, level, e, D);
  ld_b(C, J, cur, level, e, b);
  const double *cLs = sc, *cRs = sc + 20 * CRF, *Bns = sc + 40 * CRF;
#pragma unroll
  for (int r = 0; r < 5; ++r)
#pragma unroll
    for (int c = 0; c <= r; ++c) {
      double v = D[5 * r + c];
      if (tr >= 0) v -= cLs[pk(r, c) * CRF + tr];
      if (tl >= 0) v -= cRs[pk(r, c) * CRF + tl];
      next.D[(size_t)pk(r, c) * next.N + mm] = v;
    }
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    double v = b[r];
    if (tr >= 0) v -= cLs[(15 + r) * CRF + tr];
    if (tl >= 0) v -= cRs[(15 + r) * CRF + tl];
    next.b[(size_t)r * next.N + mm] = v;
  }
#pragma unroll
  for (int i = 0; i < 25; ++i) next.B[(size_t)i * next.N + mm] = tr >= 0 ? Bns[i * CRF + tr] : 0.0;
}

__global__ void __launch_bounds__(CRF) k_cr_level(DevChain C, DevJoints J, CRLevel cur, int level,
                                                  CRLevel next, int *status) {
  __shared__ double sc[65 * CRF];  // cL (20), cR (20), Bn (25) per thread
  const int t = threadIdx.x;
  const int N = cur.N, Nh = N / 2;
  const int m = blockIdx.x * (CRF - 1) + t;
  const bool have = m < Nh;
  if (have) reduce_any(C, J, cur, level, 2 * m + 1, m, Nh, sc, t, status, t < CRF - 1);
  __syncthreads();
  // even row 2m+2 (next row m+1): left odd m = thread t, right odd m+1 = thread t+1
  if (have && t < CRF - 1 && 2 * m + 2 < N) {
    const bool right = m + 1 < Nh;
    combine_row(C, J, cur, level, next, m + 1, sc, t, right ? t + 1 : -1);
  }
  // row 0 of the next level: only the odd row 1 on its right
  if (blockIdx.x == 0 && t == 0) combine_row(C, J, cur, level, next, 0, sc, -1, Nh > 0 ? 0 : -1);
}

// Back-substitution: even rows copy from the next level, odd rows solve
// lambda_n = L^{-T}(y - Ya lambda_{n-1} - Yb lambda_{n+1}).
template <int CN, int CL, int CR>
__device__ __forceinline__ void back_row(const CRLevel &cur, const CRLevel &next, int n, double *out,
                                         int out_N, int out_off, double *acc) {
  const int N = cur.N, m = (n - 1) / 2, Nh = N / 2;
  const double *f = cur.fac;
  double lL[5], lR[5], v[CN], x[CN];
#pragma unroll
  for (int r = 0; r < CL; ++r) lL[r] = next.lam[(size_t)r * next.N + m];
#pragma unroll
  for (int r = 0; r < CR; ++r) lR[r] = next.lam[(size_t)r * next.N + m + 1];
#pragma unroll
  for (int r = 0; r < CN; ++r) {
    double s = f[(size_t)(65 + r) * Nh + m];
#pragma unroll
    for (int c = 0; c < CL; ++c) s -= f[(size_t)(15 + 5 * r + c) * Nh + m] * lL[c];
#pragma unroll
    for (int c = 0; c < CR; ++c) s -= f[(size_t)(40 + 5 * r + c) * Nh + m] * lR[c];
    v[r] = s;
  }
  // L^T x = v with L packed (reciprocal diagonal)
#pragma unroll
  for (int i = CN - 1; i >= 0; --i) {
    double s = v[i];
#pragma unroll
    for (int k = i + 1; k < CN; ++k) s -= f[(size_t)pk(k, i) * Nh + m] * x[k];
    x[i] = s * f[(size_t)pk(i, i) * Nh + m];
  }
  if (n < out_off) return;
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const size_t o = (size_t)r * out_N + (n - out_off);
    const double v = r < CN ? x[r] : 0.0;
    out[o] = v;
    if (acc) acc[o] += v;
  }
}

__global__ void __launch_bounds__(128) k_cr_back(CRLevel cur, CRLevel next, DevChain C, DevJoints J,
                                                 int level, double *acc) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = cur.N;
  if (n >= N) return;
  // level 0 writes joint n - off of the chain; other levels their own rows
  double *out = level == 0 ? J.lambda : cur.lam;
  const int out_N = level == 0 ? J.K : N, out_off = level == 0 ? C.off : 0;
  if (level != 0) acc = nullptr;
  if ((n & 1) == 0) {
    if (n < out_off) return;
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      const size_t o = (size_t)r * out_N + (n - out_off);
      const double v = next.lam[(size_t)r * next.N + n / 2];
      out[o] = v;
      if (acc) acc[o] += v;
    }
    return;
  }
  const int cn = row_size(C, J, level, n), cl = row_size(C, J, level, n - 1);
  const int cr = n + 1 < N ? row_size(C, J, level, n + 1) : 0;
  const int code = (cn == 5 ? 9 : 0) + (cl == 5 ? 3 : 0) + (cr == 5 ? 2 : (cr == 3 ? 1 : 0));
  switch (code) {
#define BCK(CODE, A, B, D_) \
  case CODE: back_row<A, B, D_>(cur, next, n, out, out_N, out_off, acc); break;
    BCK(0, 3, 3, 0) BCK(1, 3, 3, 3) BCK(2, 3, 3, 5)
    BCK(3, 3, 5, 0) BCK(4, 3, 5, 3) BCK(5, 3, 5, 5)
    BCK(9, 5, 3, 0) BCK(10, 5, 3, 3) BCK(11, 5, 3, 5)
    BCK(12, 5, 5, 0) BCK(13, 5, 5, 3) BCK(14, 5, 5, 5)
#undef BCK
    default: break;
  }
}

// ---------------------------------------------------------------------------
// small levels: one warp per eliminated row
// ---------------------------------------------------------------------------
// On this GPU a warp-wide FP64 instruction occupies the warp for tens of
// cycles whatever the number of active lanes, so a level with few rows costs
// (FP64 instructions of one row) x (that latency).  The kernels below spread
// the work of a row over the lanes: every lane factors the (at most 5x5)
// diagonal block, lane c solves right-hand-side column c, and the Schur
// entries are dealt out over the lanes.

// single entries of the level's arrays (level 0 assembles them as ld_D/ld_B/ld_b do)
__device__ __forceinline__ double ldD1(const DevChain &C, const DevJoints &J, const CRLevel &L,
                                       int level, int n, int i) {
  if (level != 0) return L.D[(size_t)i * L.N + n];
  const int k = n - C.off;
  const bool diag = i == 0 || i == 2 || i == 5 || i == 9 || i == 14;
  if (k < 0) return diag ? 1.0 : 0.0;
  if (J.type[k] == 0 && (i == 9 || i == 14)) return 1.0;
  const uint8_t f = C.jflags[k];
  double v = 0.0;
  if (f & 1) v += C.Dfirst[(size_t)i * C.K + k];
  if (f & 2) v += C.Dsecond[(size_t)i * C.K + k];
  return v;
}

__device__ __forceinline__ double ldB1(const DevChain &C, const CRLevel &L, int level, int n, int i) {
  if (level != 0) return L.B[(size_t)i * L.N + n];
  const int k = n - C.off;
  return (k >= 0 && (C.jflags[k] & 4)) ? C.B[(size_t)i * C.K + k] : 0.0;
}

__device__ __forceinline__ double ldb1(const DevChain &C, const DevJoints &J, const CRLevel &L,
                                       int level, int n, int r) {
  if (level != 0) return L.b[(size_t)r * L.N + n];
  const int k = n - C.off;
  if (k < 0) return 0.0;
  const int Cs = J.type[k] == 0 ? 3 : 5;
  return r < Cs ? J.b[(size_t)r * J.K + k] : 0.0;
}

// per-warp shared workspace of one eliminated row
struct WRow {
  double D[15];       // packed diagonal block
  double Z[5][11];    // right-hand sides [B_{n-1}^T | B_n | b], then Y = L^{-1} Z
  double cl[20];      // contribution to the left row: packed -Ya^T Ya (15), -Ya^T y (5) (stored positive)
  double cr[20];      // ... to the right row
  double bn[25];      // new coupling -Ya^T Yb
};

// Cholesky with reciprocal diagonal of the packed n x n block (every lane)
__device__ __forceinline__ bool chol_rd(const double *Dp, int cn, double L[5][5], double id[5]) {
  bool ok = true;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    double sum = Dp[pk(c, c)];
#pragma unroll
    for (int k = 0; k < c; ++k) sum -= L[c][k] * L[c][k];
    if (c < cn && !(sum > 0.0)) ok = false;
    if (!(sum > 0.0)) sum = 1.0;  // rows beyond cn (and a failed pivot) get a harmless 1
    id[c] = rsqrt(sum);
    L[c][c] = sum * id[c];
#pragma unroll
    for (int r = c + 1; r < 5; ++r) {
      double t = r < cn ? Dp[pk(r, c)] : 0.0;
#pragma unroll
      for (int k = 0; k < c; ++k) t -= L[r][k] * L[c][k];
      L[r][c] = t * id[c];
    }
  }
  return ok;
}

// eliminate odd row n (index m) with one warp; fills w (contributions) and,
// when write_fac, the factor record of the row
__device__ __forceinline__ void warp_reduce_row(const DevChain &C, const DevJoints &J,
                                                const CRLevel &cur, int level, int n, int m,
                                                WRow &w, bool write_fac, int *status) {
  const int lane = threadIdx.x & 31;
  const int N = cur.N, Nh = N / 2;
  const int cn = row_size(C, J, level, n), cl = row_size(C, J, level, n - 1);
  const int cr = n + 1 < N ? row_size(C, J, level, n + 1) : 0;
  const int ncol = cl + cr + 1;
  if (lane < 15) w.D[lane] = ldD1(C, J, cur, level, n, lane);
  for (int e = lane; e < 55; e += 32) (&w.Z[0][0])[e] = 0.0;
  __syncwarp();
  if (lane < 25) {
    const int r = lane / 5, c = lane % 5;
    // B_{n-1} (cl x cn): column r of the first block of Z is its row r
    if (r < cl && c < cn) w.Z[c][r] = ldB1(C, cur, level, n - 1, lane);
    if (r < cn && c < cr) w.Z[r][cl + c] = ldB1(C, cur, level, n, lane);
  }
  if (lane < cn) w.Z[lane][cl + cr] = ldb1(C, J, cur, level, n, lane);
  __syncwarp();
  double L[5][5], id[5];
  const bool ok = chol_rd(w.D, cn, L, id);
  if (!ok && lane == 0) set_status(status, ST_NOT_SPD);
  // packed L with reciprocal diagonal (selected with constant indices so L
  // stays in registers); replaces D in the workspace
  double lp = 0.0;
#pragma unroll
  for (int r = 0; r < 5; ++r)
#pragma unroll
    for (int c = 0; c <= r; ++c)
      if (lane == r * (r + 1) / 2 + c && r < cn) lp = r == c ? id[r] : L[r][c];
  __syncwarp();
  if (lane < 15) w.D[lane] = lp;
  // lane c: column c of Y = L^{-1} Z
  double y[5];
  if (lane < ncol) {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      double t = i < cn ? w.Z[i][lane] : 0.0;
#pragma unroll
      for (int k = 0; k < i; ++k) t -= L[i][k] * y[k];
      y[i] = t * id[i];
    }
  }
  __syncwarp();
  if (lane < ncol) {
#pragma unroll
    for (int i = 0; i < 5; ++i)
      if (i < cn) w.Z[i][lane] = y[i];
  }
  __syncwarp();
  if (write_fac) {
    double *f = cur.fac;
    for (int o = lane; o < 70; o += 32) {
      double v = 0.0;
      if (o < 15) {
        v = w.D[o];
      } else if (o < 40) {
        const int r = (o - 15) / 5, c = (o - 15) % 5;
        if (r < cn && c < cl) v = w.Z[r][c];
      } else if (o < 65) {
        const int r = (o - 40) / 5, c = (o - 40) % 5;
        if (r < cn && c < cr) v = w.Z[r][cl + c];
      } else {
        const int r = o - 65;
        if (r < cn) v = w.Z[r][cl + cr];
      }
      f[(size_t)o * Nh + m] = v;
    }
  }
  // Schur entries: 0-14 Ya^T Ya packed, 15-19 Ya^T y, 20-34 Yb^T Yb packed,
  // 35-39 Yb^T y, 40-64 Ya^T Yb
  for (int e = lane; e < 65; e += 32) {
    int a = -1, b = -1;    // Z columns of the two factors
    double *dst;
    bool neg = false;
    if (e < 15 || (e >= 20 && e < 35)) {
      const int o = e < 15 ? e : e - 20;
      int r = 0;
      while ((r + 1) * (r + 2) / 2 <= o) ++r;
      const int c = o - r * (r + 1) / 2;
      if (e < 15) {
        if (r < cl && c < cl) { a = r; b = c; }
        dst = &w.cl[o];
      } else {
        if (r < cr && c < cr) { a = cl + r; b = cl + c; }
        dst = &w.cr[o];
      }
    } else if (e < 20) {
      const int r = e - 15;
      if (r < cl) { a = r; b = cl + cr; }
      dst = &w.cl[e];
    } else if (e < 40) {
      const int r = e - 35;
      if (r < cr) { a = cl + r; b = cl + cr; }
      dst = &w.cr[15 + r];
    } else {
      const int r = (e - 40) / 5, c = (e - 40) % 5;
      if (r < cl && c < cr) { a = r; b = cl + c; }
      dst = &w.bn[e - 40];
      neg = true;
    }
    double t = 0.0;
    if (a >= 0) {
#pragma unroll
      for (int i = 0; i < 5; ++i)
        if (i < cn) t += w.Z[i][a] * w.Z[i][b];
    }
    *dst = neg ? -t : t;
  }
}

// next-level row mm from even row e: D_e - (right part of the odd row on its
// left) - (left part of the odd row on its right); B from the right odd row
__device__ __forceinline__ void warp_combine_row(const DevChain &C, const DevJoints &J,
                                                 const CRLevel &cur, int level, const CRLevel &next,
                                                 int mm, const WRow *left, const WRow *right) {
  const int lane = threadIdx.x & 31;
  const int e = 2 * mm;
  for (int o = lane; o < 45; o += 32) {
    if (o < 15) {
      double v = ldD1(C, J, cur, level, e, o);
      if (right) v -= right->cl[o];
      if (left) v -= left->cr[o];
      next.D[(size_t)o * next.N + mm] = v;
    } else if (o < 20) {
      const int r = o - 15;
      double v = ldb1(C, J, cur, level, e, r);
      if (right) v -= right->cl[15 + r];
      if (left) v -= left->cr[15 + r];
      next.b[(size_t)r * next.N + mm] = v;
    } else {
      next.B[(size_t)(o - 20) * next.N + mm] = right ? right->bn[o - 20] : 0.0;
    }
  }
}

// One level: block b owns odd rows m in [b RW, b RW + RW) (warps 0..RW-1) and
// redoes odd row b RW + RW in warp RW (halo, no factor write), then forms the
// next-level rows m + 1 of its own rows (block 0 also row 0).
constexpr int RW = 4;

__global__ void __launch_bounds__(32 * (RW + 1)) k_cr_level_w(DevChain C, DevJoints J, CRLevel cur,
                                                              int level, CRLevel next, int *status) {
  __shared__ WRow ws[RW + 1];
  const int wi = threadIdx.x >> 5;
  const int N = cur.N, Nh = N / 2;
  const int m = blockIdx.x * RW + wi;
  const bool have = m < Nh;
  if (have) warp_reduce_row(C, J, cur, level, 2 * m + 1, m, ws[wi], wi < RW, status);
  __syncthreads();
  if (wi < RW && have && 2 * m + 2 < N) {
    const bool right = m + 1 < Nh;
    warp_combine_row(C, J, cur, level, next, m + 1, &ws[wi], right ? &ws[wi + 1] : nullptr);
  }
  if (blockIdx.x == 0 && wi == 0) warp_combine_row(C, J, cur, level, next, 0, nullptr, &ws[0]);
}

// Back-substitution with one warp per odd row 2m+1 (lanes r < C_n form
// v_r = y_r - Ya lambda_{n-1} - Yb lambda_{n+1}, then every lane solves
// L^T x = v); the same warp copies even row 2m from the next level.
__global__ void __launch_bounds__(128) k_cr_back_w(CRLevel cur, CRLevel next, DevChain C, DevJoints J,
                                                   int level, double *acc) {
  const int lane = threadIdx.x & 31;
  const int m = blockIdx.x * 4 + (threadIdx.x >> 5);
  const int N = cur.N, Nh = N / 2;
  if (m >= (N + 1) / 2) return;
  double *out = level == 0 ? J.lambda : cur.lam;
  const int out_N = level == 0 ? J.K : N, out_off = level == 0 ? C.off : 0;
  if (level != 0) acc = nullptr;
  {
    const int n = 2 * m;
    if (lane < 5 && n >= out_off) {
      const size_t o = (size_t)lane * out_N + (n - out_off);
      const double v = next.lam[(size_t)lane * next.N + m];
      out[o] = v;
      if (acc) acc[o] += v;
    }
  }
  if (m >= Nh) return;
  const int n = 2 * m + 1;
  const int cn = row_size(C, J, level, n), cl = row_size(C, J, level, n - 1);
  const int cr = n + 1 < N ? row_size(C, J, level, n + 1) : 0;
  const double *f = cur.fac;
  double v = 0.0;
  if (lane < cn) {
    v = f[(size_t)(65 + lane) * Nh + m];
#pragma unroll
    for (int c = 0; c < 5; ++c)
      if (c < cl) v -= f[(size_t)(15 + 5 * lane + c) * Nh + m] * next.lam[(size_t)c * next.N + m];
#pragma unroll
    for (int c = 0; c < 5; ++c)
      if (c < cr) v -= f[(size_t)(40 + 5 * lane + c) * Nh + m] * next.lam[(size_t)c * next.N + m + 1];
  }
  double vv[5], x[5];
#pragma unroll
  for (int r = 0; r < 5; ++r) vv[r] = __shfl_sync(0xffffffffu, v, r);
  // L^T x = v with L packed (reciprocal diagonal), every lane
#pragma unroll
  for (int i = 4; i >= 0; --i) {
    if (i >= cn) {
      x[i] = 0.0;
      continue;
    }
    double t = vv[i];
#pragma unroll
    for (int k = i + 1; k < 5; ++k)
      if (k < cn) t -= f[(size_t)pk(k, i) * Nh + m] * x[k];
    x[i] = t * f[(size_t)pk(i, i) * Nh + m];
  }
  if (lane < 5 && n >= out_off) {
    double xv = 0.0;
#pragma unroll
    for (int r = 0; r < 5; ++r)
      if (r == lane) xv = x[r];
    const size_t o = (size_t)lane * out_N + (n - out_off);
    out[o] = xv;
    if (acc) acc[o] += xv;
  }
}

// Single remaining row: lambda = D^{-1} b (Cholesky with reciprocal diagonal).
__global__ void k_cr_top(DevChain C, DevJoints J, CRLevel top, int level, int *status, double *acc) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const int cn = row_size(C, J, level, 0);
  double Dp[15], b[5], L[5][5], id[5], y[5], x[5];
#pragma unroll
  for (int i = 0; i < 15; ++i) Dp[i] = ldD1(C, J, top, level, 0, i);
#pragma unroll
  for (int r = 0; r < 5; ++r) b[r] = ldb1(C, J, top, level, 0, r);
  if (!chol_rd(Dp, cn, L, id)) set_status(status, ST_NOT_SPD);
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    y[i] = 0.0;
    if (i >= cn) continue;
    double t = b[i];
#pragma unroll
    for (int k = 0; k < i; ++k) t -= L[i][k] * y[k];
    y[i] = t * id[i];
  }
#pragma unroll
  for (int i = 4; i >= 0; --i) {
    x[i] = 0.0;
    if (i >= cn) continue;
    double t = y[i];
#pragma unroll
    for (int k = i + 1; k < 5; ++k)
      if (k < cn) t -= L[k][i] * x[k];
    x[i] = t * id[i];
  }
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    top.lam[(size_t)r * top.N] = x[r];
    if (acc) acc[(size_t)r * top.N] += x[r];
  }
}

// ---------------------------------------------------------------------------
// a new right-hand side through the stored factors
// ---------------------------------------------------------------------------
// y = L^{-1} b for odd row m (factor record: packed L with reciprocal diagonal)
template <int CO>
__device__ __forceinline__ void rhs_y(const double *f, int Nh, int m, const double b[5], double y[5]) {
#pragma unroll
  for (int i = 0; i < CO; ++i) {
    double t = b[i];
#pragma unroll
    for (int k = 0; k < i; ++k) t -= f[(size_t)pk(i, k) * Nh + m] * y[k];
    y[i] = t * f[(size_t)pk(i, i) * Nh + m];
  }
}

// be -= Y^T y with Y (CO x CE) the record's block at `slot` (15: Ya, 40: Yb)
template <int CO, int CE>
__device__ __forceinline__ void rhs_sub(const double *f, int Nh, int m, int slot, const double y[5],
                                        double be[5]) {
#pragma unroll
  for (int c = 0; c < CE; ++c) {
    double t = 0.0;
#pragma unroll
    for (int r = 0; r < CO; ++r) t += f[(size_t)(slot + 5 * r + c) * Nh + m] * y[r];
    be[c] -= t;
  }
}

template <int CO>
__device__ __forceinline__ void rhs_odd(const double *f, int Nh, int m, int slot, const double bo[5],
                                        int ce, double be[5], double y[5]) {
  rhs_y<CO>(f, Nh, m, bo, y);
  if (ce == 5) rhs_sub<CO, 5>(f, Nh, m, slot, y, be);
  else rhs_sub<CO, 3>(f, Nh, m, slot, y, be);
}

// One thread per next-level row mm (even row e = 2 mm): the odd rows beside
// it give y = L^{-1} b (the right one stores its y in its factor record for
// the back-substitution) and next.b[mm] = b_e - Yb_{e-1}^T y_{e-1} - Ya_{e+1}^T y_{e+1}.
__global__ void __launch_bounds__(128) k_cr_rhs(DevChain C, DevJoints J, CRLevel cur, int level,
                                                CRLevel next) {
  const int mm = blockIdx.x * blockDim.x + threadIdx.x;
  if (mm >= next.N) return;
  const int N = cur.N, Nh = N / 2, e = 2 * mm;
  const int ce = row_size(C, J, level, e);
  double be[5], bo[5], y[5];
  ld_b(C, J, cur, level, e, be);
  if (e >= 1) {  // odd row e-1 (index mm-1): its Yb couples it to e
    const int co = row_size(C, J, level, e - 1);
    ld_b(C, J, cur, level, e - 1, bo);
    if (co == 5) rhs_odd<5>(cur.fac, Nh, mm - 1, 40, bo, ce, be, y);
    else rhs_odd<3>(cur.fac, Nh, mm - 1, 40, bo, ce, be, y);
  }
  if (e + 1 < N) {  // odd row e+1 (index mm): its Ya couples it to e
    const int co = row_size(C, J, level, e + 1);
    ld_b(C, J, cur, level, e + 1, bo);
    if (co == 5) rhs_odd<5>(cur.fac, Nh, mm, 15, bo, ce, be, y);
    else rhs_odd<3>(cur.fac, Nh, mm, 15, bo, ce, be, y);
#pragma unroll
    for (int r = 0; r < 5; ++r) cur.fac[(size_t)(65 + r) * Nh + mm] = r < co ? y[r] : 0.0;
  }
#pragma unroll
  for (int r = 0; r < 5; ++r) next.b[(size_t)r * next.N + mm] = r < ce ? be[r] : 0.0;
}

static inline int nblk(int n, int t) { return (n + t - 1) / t; }

void launch_chain_gram(const DevBodies &B, const DevJoints &J, const DevIncidence &I,
                       const DevChain &C, cudaStream_t s) {
  if (B.M > 0) k_chain_gram<<<nblk(B.M, 128), 128, 0, s>>>(B, J, I, C);
}

void launch_cr_reduce(const DevChain &C, const DevJoints &J, const CRLevel &cur, int level,
                      double *cL, double *cR, double *Bn, int *status, cudaStream_t s) {
  const int Nh = cur.N / 2;
  if (Nh > 0) k_cr_reduce<<<nblk(Nh, 128), 128, 0, s>>>(C, J, cur, level, cL, cR, Bn, status);
}

void launch_cr_combine(const DevChain &C, const DevJoints &J, const CRLevel &cur, int level,
                       const CRLevel &next, const double *cL, const double *cR,
                       const double *Bn, cudaStream_t s) {
  if (next.N > 0) k_cr_combine<<<nblk(next.N, 128), 128, 0, s>>>(C, J, cur, level, next, cL, cR, Bn);
}

// levels with at most this many eliminations use one warp per row
constexpr int CR_WARP_ROWS = 2048;

void launch_cr_level(const DevChain &C, const DevJoints &J, const CRLevel &cur, int level,
                     const CRLevel &next, int *status, cudaStream_t s) {
  const int Nh = cur.N / 2;
  if (Nh >= 1 && Nh <= CR_WARP_ROWS) {
    k_cr_level_w<<<(Nh + RW - 1) / RW, 32 * (RW + 1), 0, s>>>(C, J, cur, level, next, status);
    return;
  }
  const int blocks = Nh > 0 ? (Nh + CRF - 2) / (CRF - 1) : 1;
  k_cr_level<<<blocks, CRF, 0, s>>>(C, J, cur, level, next, status);
}

void launch_cr_top(const DevChain &C, const DevJoints &J, const CRLevel &top, int level,
                   int *status, cudaStream_t s, double *acc) {
  k_cr_top<<<1, 32, 0, s>>>(C, J, top, level, status, acc);
}

void launch_cr_back(const DevChain &C, const DevJoints &J, const CRLevel &cur, const CRLevel &next,
                    int level, cudaStream_t s, double *acc) {
  if (cur.N <= 0) return;
  if (cur.N / 2 <= CR_WARP_ROWS) {
    const int rows = (cur.N + 1) / 2;
    k_cr_back_w<<<(rows + 3) / 4, 128, 0, s>>>(cur, next, C, J, level, acc);
    return;
  }
  k_cr_back<<<nblk(cur.N, 128), 128, 0, s>>>(cur, next, C, J, level, acc);
}

void launch_cr_rhs(const DevChain &C, const DevJoints &J, const CRLevel &cur, int level,
                   const CRLevel &next, cudaStream_t s) {
  if (next.N > 0) k_cr_rhs<<<nblk(next.N, 128), 128, 0, s>>>(C, J, cur, level, next);
}

void launch_mx_chain_gram(const DevBodies &B, const DevJoints &J, const DevIncidence &I,
                          const DevChain &C, cudaStream_t s) {
  if (B.M > 0) k_mx_chain_gram<<<nblk(B.M, 128), 128, 0, s>>>(B, J, I, C);
}

}  // namespace mabd
