// Block cyclic reduction of the chain's block-tridiagonal dual (Eq.
// chain-btd), templated on the arithmetic and storage type T of the
// reduction: double for the FP64 and mixed forms, float for the mixed form
// with an FP32 reduction (refined in FP64 by the correction sweeps).
// Level 0 reads the per-body Gram parts of the right precision (CRS<T>) and
// the FP64 rhs J.b; the multipliers of level 0 are written to FP64 arrays.
#pragma once
#include "mabd_device.cuh"

namespace mabd {

__device__ __forceinline__ int pk(int r, int c) { return r >= c ? r * (r + 1) / 2 + c : c * (c + 1) / 2 + r; }


// the per-body Gram parts of level 0 in the reduction's precision
template <typename T> struct CRS;
template <> struct CRS<double> {
  __device__ static const double *Df(const DevChain &C) { return C.Dfirst; }
  __device__ static const double *Ds(const DevChain &C) { return C.Dsecond; }
  __device__ static const double *Bc(const DevChain &C) { return C.B; }
};
template <> struct CRS<float> {
  __device__ static const float *Df(const DevChain &C) { return C.Dfirst_f; }
  __device__ static const float *Ds(const DevChain &C) { return C.Dsecond_f; }
  __device__ static const float *Bc(const DevChain &C) { return C.B_f; }
};

// a row of multipliers: level 0 into the FP64 output (and its accumulator),
// other levels into the level's own array
template <typename T>
__device__ __forceinline__ void cr_put(double *out64, T *outT, size_t o, T v, double *acc) {
  if (out64) {
    const double v64 = to_f64(v);
    out64[o] = v64;
    if (acc) acc[o] += v64;
  } else {
    outT[o] = v;
  }
}

// level loaders (level 0 assembles from the per-body parts; its row n is
// joint n - C.off, and a row before the first joint is a decoupled identity
// row whose multiplier is zero)
template <typename T>
__device__ __forceinline__ void ld_D(const DevChain &C, const DevJoints &J, const CRLevelT<T> &L,
                                     int level, int n, T D[25]) {
  T p[15];
  if (level == 0) {
    const int k = n - C.off;
    if (k < 0) {
#pragma unroll
      for (int i = 0; i < 15; ++i) p[i] = T(0);
#pragma unroll
      for (int r = 0; r < 5; ++r) p[pk(r, r)] = T(1);
    } else {
      const uint8_t f = C.jflags[k];
#pragma unroll
      for (int i = 0; i < 15; ++i) {
        T v = T(0);
        if (f & 1) v += CRS<T>::Df(C)[(size_t)i * C.K + k];
        if (f & 2) v += CRS<T>::Ds(C)[(size_t)i * C.K + k];
        p[i] = v;
      }
      if (J.type[k] == 0) {
        p[pk(3, 3)] = T(1);
        p[pk(4, 4)] = T(1);
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

template <typename T>
__device__ __forceinline__ void ld_B(const DevChain &C, const CRLevelT<T> &L, int level, int n,
                                     T Bm[25]) {
  if (level == 0) {
    const int k = n - C.off;
    const bool has = k >= 0 && (C.jflags[k] & 4);
#pragma unroll
    for (int i = 0; i < 25; ++i) Bm[i] = has ? CRS<T>::Bc(C)[(size_t)i * C.K + k] : T(0);
  } else {
#pragma unroll
    for (int i = 0; i < 25; ++i) Bm[i] = L.B[(size_t)i * L.N + n];
  }
}

template <typename T>
__device__ __forceinline__ void ld_b(const DevChain &C, const DevJoints &J, const CRLevelT<T> &L,
                                     int level, int n, T b[5]) {
  if (level == 0) {
    const int k = n - C.off;
    const int Cs = k < 0 ? 0 : (J.type[k] == 0 ? 3 : 5);
#pragma unroll
    for (int r = 0; r < 5; ++r) b[r] = r < Cs ? from_f64<T>(J.b[(size_t)r * J.K + k]) : T(0);
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

template <typename T, int CN, int CL, int CR>
__device__ __forceinline__ void reduce_row(const DevChain &C, const DevJoints &J, const CRLevelT<T> &cur,
                                           int level, int n, int m, int Nh, T *cL, T *cR,
                                           T *Bn, int *status, size_t cstride = 0, int cidx = -1,
                                           bool write_fac = true) {
  // contributions go to cL/cR/Bn[(i) * cstride + cidx]; by default the
  // global arrays of the level ([i][Nh], index m)
  if (cstride == 0) {
    cstride = (size_t)Nh;
    cidx = m;
  }
  // D_n, B_{n-1} (CL x CN), B_n (CN x CR), b_n
  T D[25], Bl[25], Br[25], bn[5];
  ld_D(C, J, cur, level, n, D);
  ld_B(C, cur, level, n - 1, Bl);
  if (CR > 0) ld_B(C, cur, level, n, Br);
  ld_b(C, J, cur, level, n, bn);
  // Cholesky with reciprocal diagonal
  T L[CN][CN], id[CN];
  bool ok = true;
#pragma unroll
  for (int c = 0; c < CN; ++c) {
    T sum = D[5 * c + c];
#pragma unroll
    for (int k = 0; k < c; ++k) sum -= L[c][k] * L[c][k];
    if (!(sum > T(0))) {
      ok = false;
      sum = T(1);
    }
    id[c] = rsq(sum);
    L[c][c] = sum * id[c];
#pragma unroll
    for (int r = c + 1; r < CN; ++r) {
      T t = D[5 * r + c];
#pragma unroll
      for (int k = 0; k < c; ++k) t -= L[r][k] * L[c][k];
      L[r][c] = t * id[c];
    }
  }
  if (!ok) set_status(status, ST_NOT_SPD);
  // Ya = L^{-1} B_{n-1}^T (CN x CL), Yb = L^{-1} B_n (CN x CR), y = L^{-1} b
  T Ya[CN][CL > 0 ? CL : 1], Yb[CN][CR > 0 ? CR : 1], y[CN];
#pragma unroll
  for (int i = 0; i < CN; ++i) {
#pragma unroll
    for (int c = 0; c < CL; ++c) {
      T t = Bl[5 * c + i];
#pragma unroll
      for (int k = 0; k < i; ++k) t -= L[i][k] * Ya[k][c];
      Ya[i][c] = t * id[i];
    }
#pragma unroll
    for (int c = 0; c < CR; ++c) {
      T t = Br[5 * i + c];
#pragma unroll
      for (int k = 0; k < i; ++k) t -= L[i][k] * Yb[k][c];
      Yb[i][c] = t * id[i];
    }
    T t = bn[i];
#pragma unroll
    for (int k = 0; k < i; ++k) t -= L[i][k] * y[k];
    y[i] = t * id[i];
  }
  T *f = cur.fac;
  if (write_fac) {
    int o = 0;
#pragma unroll
    for (int r = 0; r < 5; ++r)
#pragma unroll
      for (int c = 0; c <= r; ++c) {
        T v = T(0);
        if (r < CN) v = (r == c) ? id[r] : L[r][c];
        f[(size_t)(o++) * Nh + m] = v;
      }
#pragma unroll
    for (int r = 0; r < 5; ++r)
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        f[(size_t)(15 + 5 * r + c) * Nh + m] = (r < CN && c < CL) ? Ya[r][c] : T(0);
        f[(size_t)(40 + 5 * r + c) * Nh + m] = (r < CN && c < CR) ? Yb[r][c] : T(0);
      }
#pragma unroll
    for (int r = 0; r < 5; ++r) f[(size_t)(65 + r) * Nh + m] = r < CN ? y[r] : T(0);
  }
  // neighbour updates: -Ya^T Ya, -Ya^T y to row n-1; -Yb^T Yb, -Yb^T y to row n+1;
  // new coupling -Ya^T Yb between them
#pragma unroll
  for (int r = 0; r < 5; ++r) {
#pragma unroll
    for (int c = 0; c <= r; ++c) {
      T sa = T(0), sb = T(0);
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
    T ta = T(0), tb = T(0);
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
      T sab = T(0);
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
template <typename T>
__device__ __forceinline__ void cr_reduce_one(DevChain C, DevJoints J, CRLevelT<T> cur, int level,
                                                   T *cL, T *cR, T *Bn, int *status, int m) {
  
  const int n = 2 * m + 1;
  const int N = cur.N;
  if (n >= N) return;
  const int Nh = N / 2;
  const int cn = row_size(C, J, level, n), cl = row_size(C, J, level, n - 1);
  const int cr = n + 1 < N ? row_size(C, J, level, n + 1) : 0;
  const int code = (cn == 5 ? 9 : 0) + (cl == 5 ? 3 : 0) + (cr == 5 ? 2 : (cr == 3 ? 1 : 0));
  switch (code) {
#define RED(CODE, A, B, D_) \
  case CODE: reduce_row<T, A, B, D_>(C, J, cur, level, n, m, Nh, cL, cR, Bn, status); break;
    RED(0, 3, 3, 0) RED(1, 3, 3, 3) RED(2, 3, 3, 5)
    RED(3, 3, 5, 0) RED(4, 3, 5, 3) RED(5, 3, 5, 5)
    RED(9, 5, 3, 0) RED(10, 5, 3, 3) RED(11, 5, 3, 5)
    RED(12, 5, 5, 0) RED(13, 5, 5, 3) RED(14, 5, 5, 5)
#undef RED
    default: break;
  }
}

template <typename T>
__global__ void __launch_bounds__(128) k_cr_reduce(DevChain C, DevJoints J, CRLevelT<T> cur, int level,
                                                   T *cL, T *cR, T *Bn, int *status) {
  cr_reduce_one<T>(C, J, cur, level, cL, cR, Bn, status, blockIdx.x * blockDim.x + threadIdx.x);
}

// Even row e = 2m becomes row m of the next level.
template <typename T>
__device__ __forceinline__ void cr_combine_one(DevChain C, DevJoints J, CRLevelT<T> cur, int level,
                                                    CRLevelT<T> next, const T *cL,
                                                    const T *cR, const T *Bn, int m) {
  
  if (m >= next.N) return;
  const int e = 2 * m;
  const int N = cur.N, Nh = N / 2;
  T D[25], b[5];
  ld_D(C, J, cur, level, e, D);
  ld_b(C, J, cur, level, e, b);
  const bool right = e + 1 < N;  // odd row e+1 exists (its index m)
  const bool left = e >= 1;      // odd row e-1 exists (its index m-1)
#pragma unroll
  for (int r = 0; r < 5; ++r)
#pragma unroll
    for (int c = 0; c <= r; ++c) {
      T v = D[5 * r + c];
      if (right) v -= cL[(size_t)pk(r, c) * Nh + m];
      if (left) v -= cR[(size_t)pk(r, c) * Nh + m - 1];
      next.D[(size_t)pk(r, c) * next.N + m] = v;
    }
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    T v = b[r];
    if (right) v -= cL[(size_t)(15 + r) * Nh + m];
    if (left) v -= cR[(size_t)(15 + r) * Nh + m - 1];
    next.b[(size_t)r * next.N + m] = v;
  }
#pragma unroll
  for (int i = 0; i < 25; ++i) next.B[(size_t)i * next.N + m] = right ? Bn[(size_t)i * Nh + m] : T(0);
}

template <typename T>
__global__ void __launch_bounds__(128) k_cr_combine(DevChain C, DevJoints J, CRLevelT<T> cur, int level,
                                                    CRLevelT<T> next, const T *cL,
                                                    const T *cR, const T *Bn) {
  cr_combine_one<T>(C, J, cur, level, next, cL, cR, Bn, blockIdx.x * blockDim.x + threadIdx.x);
}

// One cyclic-reduction level in one launch.  Block b owns the odd rows
// m in [b*(CRF-1), (b+1)*(CRF-1)); its last thread redoes the first odd row
// of the next block as a halo (no factor write).  After the eliminations the
// contributions meet in shared memory and thread t forms next-level row
// m+1 (even row 2m+2) from its own right contribution and the left
// contribution and new coupling of thread t+1; block 0 also forms row 0.
constexpr int CRF = 64;

template <typename T, int CN, int CL, int CR>
__device__ __forceinline__ void reduce_row_s(const DevChain &C, const DevJoints &J, const CRLevelT<T> &cur,
                                             int level, int n, int m, int Nh, T *sc, int t,
                                             int *status, bool write_fac) {
  reduce_row<T, CN, CL, CR>(C, J, cur, level, n, m, Nh, sc, sc + 20 * CRF, sc + 40 * CRF, status,
                         (size_t)CRF, t, write_fac);
}

template <typename T>
__device__ __forceinline__ void reduce_any(const DevChain &C, const DevJoints &J, const CRLevelT<T> &cur,
                                           int level, int n, int m, int Nh, T *sc, int t,
                                           int *status, bool write_fac) {
  const int N = cur.N;
  const int cn = row_size(C, J, level, n), cl = row_size(C, J, level, n - 1);
  const int cr = n + 1 < N ? row_size(C, J, level, n + 1) : 0;
  const int code = (cn == 5 ? 9 : 0) + (cl == 5 ? 3 : 0) + (cr == 5 ? 2 : (cr == 3 ? 1 : 0));
  switch (code) {
#define RED(CODE, A, B_, D_) \
  case CODE: reduce_row_s<T, A, B_, D_>(C, J, cur, level, n, m, Nh, sc, t, status, write_fac); break;
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
template <typename T>
__device__ __forceinline__ void combine_row(const DevChain &C, const DevJoints &J, const CRLevelT<T> &cur,
                                            int level, const CRLevelT<T> &next, int mm, const T *sc,
                                            int tl, int tr) {
  const int e = 2 * mm;
  T D[25], b[5];
  ld_D(C, J, cur, level, e, D);
  ld_b(C, J, cur, level, e, b);
  const T *cLs = sc, *cRs = sc + 20 * CRF, *Bns = sc + 40 * CRF;
#pragma unroll
  for (int r = 0; r < 5; ++r)
#pragma unroll
    for (int c = 0; c <= r; ++c) {
      T v = D[5 * r + c];
      if (tr >= 0) v -= cLs[pk(r, c) * CRF + tr];
      if (tl >= 0) v -= cRs[pk(r, c) * CRF + tl];
      next.D[(size_t)pk(r, c) * next.N + mm] = v;
    }
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    T v = b[r];
    if (tr >= 0) v -= cLs[(15 + r) * CRF + tr];
    if (tl >= 0) v -= cRs[(15 + r) * CRF + tl];
    next.b[(size_t)r * next.N + mm] = v;
  }
#pragma unroll
  for (int i = 0; i < 25; ++i) next.B[(size_t)i * next.N + mm] = tr >= 0 ? Bns[i * CRF + tr] : T(0);
}

template <typename T>
__global__ void __launch_bounds__(CRF) k_cr_level(DevChain C, DevJoints J, CRLevelT<T> cur, int level,
                                                  CRLevelT<T> next, int *status) {
  __shared__ T sc[65 * CRF];  // cL (20), cR (20), Bn (25) per thread
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
template <typename T, int CN, int CL, int CR>
__device__ __forceinline__ void back_row(const CRLevelT<T> &cur, const CRLevelT<T> &next, int n,
                                         double *out64, T *outT, int out_N, int out_off, double *acc) {
  const int N = cur.N, m = (n - 1) / 2, Nh = N / 2;
  const T *f = cur.fac;
  T lL[5], lR[5], v[CN], x[CN];
#pragma unroll
  for (int r = 0; r < CL; ++r) lL[r] = next.lam[(size_t)r * next.N + m];
#pragma unroll
  for (int r = 0; r < CR; ++r) lR[r] = next.lam[(size_t)r * next.N + m + 1];
#pragma unroll
  for (int r = 0; r < CN; ++r) {
    T s = f[(size_t)(65 + r) * Nh + m];
#pragma unroll
    for (int c = 0; c < CL; ++c) s -= f[(size_t)(15 + 5 * r + c) * Nh + m] * lL[c];
#pragma unroll
    for (int c = 0; c < CR; ++c) s -= f[(size_t)(40 + 5 * r + c) * Nh + m] * lR[c];
    v[r] = s;
  }
  // L^T x = v with L packed (reciprocal diagonal)
#pragma unroll
  for (int i = CN - 1; i >= 0; --i) {
    T s = v[i];
#pragma unroll
    for (int k = i + 1; k < CN; ++k) s -= f[(size_t)pk(k, i) * Nh + m] * x[k];
    x[i] = s * f[(size_t)pk(i, i) * Nh + m];
  }
  if (n < out_off) return;
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const size_t o = (size_t)r * out_N + (n - out_off);
    cr_put(out64, outT, o, r < CN ? x[r] : T(0), acc);
  }
}

template <typename T>
__device__ __forceinline__ void cr_back_one(CRLevelT<T> cur, CRLevelT<T> next, DevChain C, DevJoints J,
                                                 int level, double *acc, int n) {
  
  const int N = cur.N;
  if (n >= N) return;
  // level 0 writes joint n - off of the chain (FP64); other levels their own rows
  double *out64 = level == 0 ? J.lambda : nullptr;
  T *outT = level == 0 ? nullptr : cur.lam;
  const int out_N = level == 0 ? J.K : N, out_off = level == 0 ? C.off : 0;
  if (level != 0) acc = nullptr;
  if ((n & 1) == 0) {
    if (n < out_off) return;
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      const size_t o = (size_t)r * out_N + (n - out_off);
      cr_put(out64, outT, o, next.lam[(size_t)r * next.N + n / 2], acc);
    }
    return;
  }
  const int cn = row_size(C, J, level, n), cl = row_size(C, J, level, n - 1);
  const int cr = n + 1 < N ? row_size(C, J, level, n + 1) : 0;
  const int code = (cn == 5 ? 9 : 0) + (cl == 5 ? 3 : 0) + (cr == 5 ? 2 : (cr == 3 ? 1 : 0));
  switch (code) {
#define BCK(CODE, A, B, D_) \
  case CODE: back_row<T, A, B, D_>(cur, next, n, out64, outT, out_N, out_off, acc); break;
    BCK(0, 3, 3, 0) BCK(1, 3, 3, 3) BCK(2, 3, 3, 5)
    BCK(3, 3, 5, 0) BCK(4, 3, 5, 3) BCK(5, 3, 5, 5)
    BCK(9, 5, 3, 0) BCK(10, 5, 3, 3) BCK(11, 5, 3, 5)
    BCK(12, 5, 5, 0) BCK(13, 5, 5, 3) BCK(14, 5, 5, 5)
#undef BCK
    default: break;
  }
}

// Back-substitution of one level with one thread per row pair: even row 2m
// (a copy from the next level) and odd row 2m+1 (the solve).  With a thread
// per row the odd and even lanes of a warp diverge and each path runs with
// half the lanes; here every lane solves, and the factor loads of a warp
// cover 32 consecutive m.
template <typename T>
__global__ void __launch_bounds__(128) k_cr_back_pair(CRLevelT<T> cur, CRLevelT<T> next, DevChain C,
                                                      DevJoints J, int level, double *acc) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * m >= cur.N) return;
  cr_back_one<T>(cur, next, C, J, level, acc, 2 * m);
  cr_back_one<T>(cur, next, C, J, level, acc, 2 * m + 1);
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
template <typename T>
__device__ __forceinline__ T ldD1(const DevChain &C, const DevJoints &J, const CRLevelT<T> &L,
                                       int level, int n, int i) {
  if (level != 0) return L.D[(size_t)i * L.N + n];
  const int k = n - C.off;
  const bool diag = i == 0 || i == 2 || i == 5 || i == 9 || i == 14;
  if (k < 0) return diag ? T(1) : T(0);
  if (J.type[k] == 0 && (i == 9 || i == 14)) return T(1);
  const uint8_t f = C.jflags[k];
  T v = T(0);
  if (f & 1) v += CRS<T>::Df(C)[(size_t)i * C.K + k];
  if (f & 2) v += CRS<T>::Ds(C)[(size_t)i * C.K + k];
  return v;
}

template <typename T>
__device__ __forceinline__ T ldB1(const DevChain &C, const CRLevelT<T> &L, int level, int n, int i) {
  if (level != 0) return L.B[(size_t)i * L.N + n];
  const int k = n - C.off;
  return (k >= 0 && (C.jflags[k] & 4)) ? CRS<T>::Bc(C)[(size_t)i * C.K + k] : T(0);
}

template <typename T>
__device__ __forceinline__ T ldb1(const DevChain &C, const DevJoints &J, const CRLevelT<T> &L,
                                       int level, int n, int r) {
  if (level != 0) return L.b[(size_t)r * L.N + n];
  const int k = n - C.off;
  if (k < 0) return T(0);
  const int Cs = J.type[k] == 0 ? 3 : 5;
  return r < Cs ? from_f64<T>(J.b[(size_t)r * J.K + k]) : T(0);
}

// per-warp shared workspace of one eliminated row
template <typename T>
struct WRow {
  T D[15];       // packed diagonal block
  T Z[5][11];    // right-hand sides [B_{n-1}^T | B_n | b], then Y = L^{-1} Z
  T cl[20];      // contribution to the left row: packed -Ya^T Ya (15), -Ya^T y (5) (stored positive)
  T cr[20];      // ... to the right row
  T bn[25];      // new coupling -Ya^T Yb
};

// Cholesky with reciprocal diagonal of the packed n x n block (every lane)
template <typename T>
__device__ __forceinline__ bool chol_rd(const T *Dp, int cn, T L[5][5], T id[5]) {
  bool ok = true;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    T sum = Dp[pk(c, c)];
#pragma unroll
    for (int k = 0; k < c; ++k) sum -= L[c][k] * L[c][k];
    if (c < cn && !(sum > T(0))) ok = false;
    if (!(sum > T(0))) sum = T(1);  // rows beyond cn (and a failed pivot) get a harmless 1
    id[c] = rsq(sum);
    L[c][c] = sum * id[c];
#pragma unroll
    for (int r = c + 1; r < 5; ++r) {
      T t = r < cn ? Dp[pk(r, c)] : T(0);
#pragma unroll
      for (int k = 0; k < c; ++k) t -= L[r][k] * L[c][k];
      L[r][c] = t * id[c];
    }
  }
  return ok;
}

// eliminate odd row n (index m) with one warp; fills w (contributions) and,
// when write_fac, the factor record of the row
template <typename T>
__device__ __forceinline__ void warp_reduce_row(const DevChain &C, const DevJoints &J,
                                                const CRLevelT<T> &cur, int level, int n, int m,
                                                WRow<T> &w, bool write_fac, int *status) {
  const int lane = threadIdx.x & 31;
  const int N = cur.N, Nh = N / 2;
  const int cn = row_size(C, J, level, n), cl = row_size(C, J, level, n - 1);
  const int cr = n + 1 < N ? row_size(C, J, level, n + 1) : 0;
  const int ncol = cl + cr + 1;
  if (lane < 15) w.D[lane] = ldD1(C, J, cur, level, n, lane);
  for (int e = lane; e < 55; e += 32) (&w.Z[0][0])[e] = T(0);
  __syncwarp();
  if (lane < 25) {
    const int r = lane / 5, c = lane % 5;
    // B_{n-1} (cl x cn): column r of the first block of Z is its row r
    if (r < cl && c < cn) w.Z[c][r] = ldB1(C, cur, level, n - 1, lane);
    if (r < cn && c < cr) w.Z[r][cl + c] = ldB1(C, cur, level, n, lane);
  }
  if (lane < cn) w.Z[lane][cl + cr] = ldb1(C, J, cur, level, n, lane);
  __syncwarp();
  T L[5][5], id[5];
  const bool ok = chol_rd(w.D, cn, L, id);
  if (!ok && lane == 0) set_status(status, ST_NOT_SPD);
  // packed L with reciprocal diagonal (selected with constant indices so L
  // stays in registers); replaces D in the workspace
  T lp = T(0);
#pragma unroll
  for (int r = 0; r < 5; ++r)
#pragma unroll
    for (int c = 0; c <= r; ++c)
      if (lane == r * (r + 1) / 2 + c && r < cn) lp = r == c ? id[r] : L[r][c];
  __syncwarp();
  if (lane < 15) w.D[lane] = lp;
  // lane c: column c of Y = L^{-1} Z
  T y[5];
  if (lane < ncol) {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      T t = i < cn ? w.Z[i][lane] : T(0);
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
    T *f = cur.fac;
    for (int o = lane; o < 70; o += 32) {
      T v = T(0);
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
    T *dst;
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
    T t = T(0);
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
template <typename T>
__device__ __forceinline__ void warp_combine_row(const DevChain &C, const DevJoints &J,
                                                 const CRLevelT<T> &cur, int level, const CRLevelT<T> &next,
                                                 int mm, const WRow<T> *left, const WRow<T> *right) {
  const int lane = threadIdx.x & 31;
  const int e = 2 * mm;
  for (int o = lane; o < 45; o += 32) {
    if (o < 15) {
      T v = ldD1(C, J, cur, level, e, o);
      if (right) v -= right->cl[o];
      if (left) v -= left->cr[o];
      next.D[(size_t)o * next.N + mm] = v;
    } else if (o < 20) {
      const int r = o - 15;
      T v = ldb1(C, J, cur, level, e, r);
      if (right) v -= right->cl[15 + r];
      if (left) v -= left->cr[15 + r];
      next.b[(size_t)r * next.N + mm] = v;
    } else {
      next.B[(size_t)(o - 20) * next.N + mm] = right ? right->bn[o - 20] : T(0);
    }
  }
}

// One level: block b owns odd rows m in [b RW, b RW + RW) (warps 0..RW-1) and
// redoes odd row b RW + RW in warp RW (halo, no factor write), then forms the
// next-level rows m + 1 of its own rows (block 0 also row 0).
constexpr int RW = 4;

template <typename T>
__global__ void __launch_bounds__(32 * (RW + 1)) k_cr_level_w(DevChain C, DevJoints J, CRLevelT<T> cur,
                                                              int level, CRLevelT<T> next, int *status) {
  __shared__ WRow<T> ws[RW + 1];
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
  if (blockIdx.x == 0 && wi == 0) warp_combine_row<T>(C, J, cur, level, next, 0, nullptr, &ws[0]);
}

// Back-substitution with one warp per odd row 2m+1 (lanes r < C_n form
// v_r = y_r - Ya lambda_{n-1} - Yb lambda_{n+1}, then every lane solves
// L^T x = v); the same warp copies even row 2m from the next level.
template <typename T>
__global__ void __launch_bounds__(128) k_cr_back_w(CRLevelT<T> cur, CRLevelT<T> next, DevChain C, DevJoints J,
                                                   int level, double *acc) {
  const int lane = threadIdx.x & 31;
  const int m = blockIdx.x * 4 + (threadIdx.x >> 5);
  const int N = cur.N, Nh = N / 2;
  if (m >= (N + 1) / 2) return;
  double *out64 = level == 0 ? J.lambda : nullptr;
  T *outT = level == 0 ? nullptr : cur.lam;
  const int out_N = level == 0 ? J.K : N, out_off = level == 0 ? C.off : 0;
  if (level != 0) acc = nullptr;
  {
    const int n = 2 * m;
    if (lane < 5 && n >= out_off) {
      const size_t o = (size_t)lane * out_N + (n - out_off);
      cr_put(out64, outT, o, next.lam[(size_t)lane * next.N + m], acc);
    }
  }
  if (m >= Nh) return;
  const int n = 2 * m + 1;
  const int cn = row_size(C, J, level, n), cl = row_size(C, J, level, n - 1);
  const int cr = n + 1 < N ? row_size(C, J, level, n + 1) : 0;
  const T *f = cur.fac;
  T v = T(0);
  if (lane < cn) {
    v = f[(size_t)(65 + lane) * Nh + m];
#pragma unroll
    for (int c = 0; c < 5; ++c)
      if (c < cl) v -= f[(size_t)(15 + 5 * lane + c) * Nh + m] * next.lam[(size_t)c * next.N + m];
#pragma unroll
    for (int c = 0; c < 5; ++c)
      if (c < cr) v -= f[(size_t)(40 + 5 * lane + c) * Nh + m] * next.lam[(size_t)c * next.N + m + 1];
  }
  T vv[5], x[5];
#pragma unroll
  for (int r = 0; r < 5; ++r) vv[r] = __shfl_sync(0xffffffffu, v, r);
  // L^T x = v with L packed (reciprocal diagonal), every lane
#pragma unroll
  for (int i = 4; i >= 0; --i) {
    if (i >= cn) {
      x[i] = T(0);
      continue;
    }
    T t = vv[i];
#pragma unroll
    for (int k = i + 1; k < 5; ++k)
      if (k < cn) t -= f[(size_t)pk(k, i) * Nh + m] * x[k];
    x[i] = t * f[(size_t)pk(i, i) * Nh + m];
  }
  if (lane < 5 && n >= out_off) {
    T xv = T(0);
#pragma unroll
    for (int r = 0; r < 5; ++r)
      if (r == lane) xv = x[r];
    const size_t o = (size_t)lane * out_N + (n - out_off);
    cr_put(out64, outT, o, xv, acc);
  }
}

// Single remaining row: lambda = D^{-1} b (Cholesky with reciprocal diagonal).
template <typename T>
__device__ __forceinline__ void cr_top_one(const DevChain &C, const DevJoints &J, const CRLevelT<T> &top,
                                           int level, int *status, double *out64, double *acc) {
  const int cn = row_size(C, J, level, 0);
  T Dp[15], b[5], L[5][5], id[5], y[5], x[5];
#pragma unroll
  for (int i = 0; i < 15; ++i) Dp[i] = ldD1(C, J, top, level, 0, i);
#pragma unroll
  for (int r = 0; r < 5; ++r) b[r] = ldb1(C, J, top, level, 0, r);
  if (!chol_rd(Dp, cn, L, id)) set_status(status, ST_NOT_SPD);
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    y[i] = T(0);
    if (i >= cn) continue;
    T t = b[i];
#pragma unroll
    for (int k = 0; k < i; ++k) t -= L[i][k] * y[k];
    y[i] = t * id[i];
  }
#pragma unroll
  for (int i = 4; i >= 0; --i) {
    x[i] = T(0);
    if (i >= cn) continue;
    T t = y[i];
#pragma unroll
    for (int k = i + 1; k < 5; ++k)
      if (k < cn) t -= L[k][i] * x[k];
    x[i] = t * id[i];
  }
#pragma unroll
  for (int r = 0; r < 5; ++r) cr_put(out64, top.lam, (size_t)r * top.N, x[r], out64 ? acc : nullptr);
}

template <typename T>
__global__ void k_cr_top(DevChain C, DevJoints J, CRLevelT<T> top, int level, int *status, double *out64,
                         double *acc) {
  if (blockIdx.x == 0 && threadIdx.x == 0) cr_top_one<T>(C, J, top, level, status, out64, acc);
}

// ---------------------------------------------------------------------------
// a new right-hand side through the stored factors
// ---------------------------------------------------------------------------
// y = L^{-1} b for odd row m (factor record: packed L with reciprocal diagonal)
template <typename T, int CO>
__device__ __forceinline__ void rhs_y(const T *f, int Nh, int m, const T b[5], T y[5]) {
#pragma unroll
  for (int i = 0; i < CO; ++i) {
    T t = b[i];
#pragma unroll
    for (int k = 0; k < i; ++k) t -= f[(size_t)pk(i, k) * Nh + m] * y[k];
    y[i] = t * f[(size_t)pk(i, i) * Nh + m];
  }
}

// be -= Y^T y with Y (CO x CE) the record's block at `slot` (15: Ya, 40: Yb)
template <typename T, int CO, int CE>
__device__ __forceinline__ void rhs_sub(const T *f, int Nh, int m, int slot, const T y[5],
                                        T be[5]) {
#pragma unroll
  for (int c = 0; c < CE; ++c) {
    T t = T(0);
#pragma unroll
    for (int r = 0; r < CO; ++r) t += f[(size_t)(slot + 5 * r + c) * Nh + m] * y[r];
    be[c] -= t;
  }
}

template <typename T, int CO>
__device__ __forceinline__ void rhs_odd(const T *f, int Nh, int m, int slot, const T bo[5],
                                        int ce, T be[5], T y[5]) {
  rhs_y<T, CO>(f, Nh, m, bo, y);
  if (ce == 5) rhs_sub<T, CO, 5>(f, Nh, m, slot, y, be);
  else rhs_sub<T, CO, 3>(f, Nh, m, slot, y, be);
}

// One thread per next-level row mm (even row e = 2 mm): the odd rows beside
// it give y = L^{-1} b (the right one stores its y in its factor record for
// the back-substitution) and next.b[mm] = b_e - Yb_{e-1}^T y_{e-1} - Ya_{e+1}^T y_{e+1}.
template <typename T>
__device__ __forceinline__ void cr_rhs_one(DevChain C, DevJoints J, CRLevelT<T> cur, int level,
                                                CRLevelT<T> next, int mm) {
  
  if (mm >= next.N) return;
  const int N = cur.N, Nh = N / 2, e = 2 * mm;
  const int ce = row_size(C, J, level, e);
  T be[5], bo[5], y[5];
  ld_b(C, J, cur, level, e, be);
  if (e >= 1) {  // odd row e-1 (index mm-1): its Yb couples it to e
    const int co = row_size(C, J, level, e - 1);
    ld_b(C, J, cur, level, e - 1, bo);
    if (co == 5) rhs_odd<T, 5>(cur.fac, Nh, mm - 1, 40, bo, ce, be, y);
    else rhs_odd<T, 3>(cur.fac, Nh, mm - 1, 40, bo, ce, be, y);
  }
  if (e + 1 < N) {  // odd row e+1 (index mm): its Ya couples it to e
    const int co = row_size(C, J, level, e + 1);
    ld_b(C, J, cur, level, e + 1, bo);
    if (co == 5) rhs_odd<T, 5>(cur.fac, Nh, mm, 15, bo, ce, be, y);
    else rhs_odd<T, 3>(cur.fac, Nh, mm, 15, bo, ce, be, y);
#pragma unroll
    for (int r = 0; r < 5; ++r) cur.fac[(size_t)(65 + r) * Nh + mm] = r < co ? y[r] : T(0);
  }
#pragma unroll
  for (int r = 0; r < 5; ++r) next.b[(size_t)r * next.N + mm] = r < ce ? be[r] : T(0);
}

template <typename T>
__global__ void __launch_bounds__(128) k_cr_rhs(DevChain C, DevJoints J, CRLevelT<T> cur, int level,
                                                CRLevelT<T> next) {
  cr_rhs_one<T>(C, J, cur, level, next, blockIdx.x * blockDim.x + threadIdx.x);
}


// ---------------------------------------------------------------------------
// the small levels in one CTA
// ---------------------------------------------------------------------------
// Levels l0 .. nl-2 (elimination or right-hand-side pass), the top row and the
// back-substitution down to level l0, with a CTA barrier between levels: the
// rows of a level are dealt out over the threads with the thread-per-row
// bodies of the multi-CTA kernels.  This replaces two launches per level with
// one launch, which pays where a row's serial latency is short (FP32) and the
// levels hold at most a few hundred rows.  cL/cR/Bn hold (20, 20, 25) x Nh of
// the largest level.
// (FP64 rows need more registers than 512 threads leave)
template <typename T>
constexpr int cr_tail_threads() { return sizeof(T) == 4 ? 512 : 256; }

template <typename T>
__global__ void __launch_bounds__(cr_tail_threads<T>()) k_cr_tail(DevChain C, DevJoints J, DevJoints Jout,
                                                             const CRLevelT<T> *lv, int l0, int nl,
                                                             int rhs_only, T *cL, T *cR, T *Bn, int *status,
                                                             double *acc) {
  const int t = threadIdx.x, nt = blockDim.x;
  for (int l = l0; l + 1 < nl; ++l) {
    const CRLevelT<T> cur = lv[l], next = lv[l + 1];
    if (rhs_only) {
      for (int mm = t; mm < next.N; mm += nt) cr_rhs_one<T>(C, J, cur, l, next, mm);
    } else {
      const int Nh = cur.N / 2;
      for (int m = t; m < Nh; m += nt) cr_reduce_one<T>(C, J, cur, l, cL, cR, Bn, status, m);
      __syncthreads();
      for (int m = t; m < next.N; m += nt) cr_combine_one<T>(C, J, cur, l, next, cL, cR, Bn, m);
    }
    __syncthreads();
  }
  if (t == 0) {
    // a single row at level 0 (one joint) is the top row and the output
    if (nl == 1) cr_top_one<T>(C, J, lv[0], 0, status, Jout.lambda, acc);
    else cr_top_one<T>(C, J, lv[nl - 1], nl - 1, status, nullptr, nullptr);
  }
  __syncthreads();
  for (int l = nl - 2; l >= l0; --l) {
    const CRLevelT<T> cur = lv[l], next = lv[l + 1];
    for (int n = t; n < cur.N; n += nt)
      cr_back_one<T>(cur, next, C, l == 0 ? Jout : J, l, l == 0 ? acc : nullptr, n);
    __syncthreads();
  }
}


}  // namespace mabd
