// Chain path of one M-ABD step, Sec. 5.2 (also the chain part of the loop
// solver, Sec. 5.4, whose closing body writes the corner block):
//   k_chain_gram  per body j: the Gram blocks of its (at most two) joints,
//                 G_kj H_j^{-1} G_k'j^T (Eq. chain-Schur-blocks), formed in the
//                 body's rest frame with the structured Hbar^{-1};
//   k_cr_*        block cyclic reduction of the block-tridiagonal dual
//                 (Eq. chain-btd, cr_impl.cuh, in FP64 or FP32) with every
//                 block padded to 5x5 (a ball's two extra rows carry an
//                 identity diagonal and decouple exactly).
// Packed lower-triangular 5x5 storage: entry (r, c), r >= c, at r(r+1)/2 + c.
#include "cr_impl.cuh"

namespace mabd {


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

template <typename T, typename HT, typename OT = double>
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
  // the slot loops run over both slots (unrolled), so that E and P stay in
  // registers; a run-time slot index would put them in local memory
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    if (s >= n) break;
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
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    if (s >= n) break;
    OT *dst = const_cast<OT *>(C.islot[e0 + s] == 0 ? CRS<OT>::Df(C) : CRS<OT>::Ds(C));
    const int k = kk[s];
    OT Dp[15];
#pragma unroll
    for (int i = 0; i < 15; ++i) Dp[i] = OT(0);
    mbar(h, P[s][0], P[s][0], Mb);
    project<3, 3>(E[s], c012, Mb, E[s], c012, blk);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c <= r; ++c) Dp[pk(r, c)] = (OT)blk[r][c];
    if (ty[s] == 1) {
      mbar(h, P[s][1], P[s][0], Mb);                      // rows 3-4 x rows 0-2
      project<2, 3>(E[s], c02, Mb, E[s], c012, blk);
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) Dp[pk(3 + r, c)] = (OT)blk[r][c];
      mbar(h, P[s][1], P[s][1], Mb);                      // rows 3-4 x rows 3-4
      project<2, 2>(E[s], c02, Mb, E[s], c02, blk);
      Dp[pk(3, 3)] = (OT)blk[0][0];
      Dp[pk(4, 3)] = (OT)blk[1][0];
      Dp[pk(4, 4)] = (OT)blk[1][1];
    }
#pragma unroll
    for (int i = 0; i < 15; ++i) dst[(size_t)i * K + k] = Dp[i];
  }
  if (n == 2) {
    // coupling of the two joints: rows of joint 0 x rows of joint 1 -> B[k0]
    OT Bp[25];
#pragma unroll
    for (int i = 0; i < 25; ++i) Bp[i] = OT(0);
    mbar(h, P[0][0], P[1][0], Mb);
    project<3, 3>(E[0], c012, Mb, E[1], c012, blk);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) Bp[5 * r + c] = (OT)blk[r][c];
    if (ty[1] == 1) {
      mbar(h, P[0][0], P[1][1], Mb);
      project<3, 2>(E[0], c012, Mb, E[1], c02, blk);
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) Bp[5 * r + 3 + c] = (OT)blk[r][c];
    }
    if (ty[0] == 1) {
      mbar(h, P[0][1], P[1][0], Mb);
      project<2, 3>(E[0], c02, Mb, E[1], c012, blk);
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) Bp[5 * (3 + r) + c] = (OT)blk[r][c];
      if (ty[1] == 1) {
        mbar(h, P[0][1], P[1][1], Mb);
        project<2, 2>(E[0], c02, Mb, E[1], c02, blk);
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
          for (int c = 0; c < 2; ++c) Bp[5 * (3 + r) + 3 + c] = (OT)blk[r][c];
      }
    }
    const int k0 = kk[0];
    if (kk[1] != k0 + 1) {
      // the body that closes a loop: joint 0 and the loop breaker K - 1
      if (C.corner && sizeof(OT) == 8)
#pragma unroll
        for (int i = 0; i < 25; ++i) C.corner[i] = (double)Bp[i];
      return;
    }
    OT *Bd = const_cast<OT *>(CRS<OT>::Bc(C));
#pragma unroll
    for (int i = 0; i < 25; ++i) Bd[(size_t)i * K + k0] = Bp[i];
  }
}

__global__ void __launch_bounds__(128) k_chain_gram(DevBodies B, DevJoints J, DevIncidence I,
                                                    DevChain C) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < B.M) chain_gram_body<double>(B, J, I, C, B.hinv, ordered(B.order, t));
}

// mixed-precision form: the same blocks with FP32 products, stored in FP64
// for the FP64 reduction or in FP32 for the FP32 one
template <typename OT>
__global__ void __launch_bounds__(128) k_mx_chain_gram(DevBodies B, DevJoints J, DevIncidence I,
                                                       DevChain C) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < B.M) chain_gram_body<float, float, OT>(B, J, I, C, B.hinvf, ordered(B.order, t));
}

static inline int nblk(int n, int t) { return (n + t - 1) / t; }

void launch_chain_gram(const DevBodies &B, const DevJoints &J, const DevIncidence &I,
                       const DevChain &C, cudaStream_t s) {
  if (B.M > 0) k_chain_gram<<<nblk(B.M, 128), 128, 0, s>>>(B, J, I, C);
}

void launch_cr_reduce(const DevChain &C, const DevJoints &J, const CRLevel &cur, int level,
                      double *cL, double *cR, double *Bn, int *status, cudaStream_t s) {
  const int Nh = cur.N / 2;
  if (Nh > 0) k_cr_reduce<double><<<nblk(Nh, 128), 128, 0, s>>>(C, J, cur, level, cL, cR, Bn, status);
}

void launch_cr_combine(const DevChain &C, const DevJoints &J, const CRLevel &cur, int level,
                       const CRLevel &next, const double *cL, const double *cR,
                       const double *Bn, cudaStream_t s) {
  if (next.N > 0) k_cr_combine<double><<<nblk(next.N, 128), 128, 0, s>>>(C, J, cur, level, next, cL, cR, Bn);
}

// levels with at most this many eliminations use one warp per row
constexpr int CR_WARP_ROWS = 2048;

template <typename T>
void launch_cr_level(const DevChain &C, const DevJoints &J, const CRLevelT<T> &cur, int level,
                     const CRLevelT<T> &next, int *status, cudaStream_t s) {
  const int Nh = cur.N / 2;
  if (Nh >= 1 && Nh <= CR_WARP_ROWS) {
    k_cr_level_w<T><<<(Nh + RW - 1) / RW, 32 * (RW + 1), 0, s>>>(C, J, cur, level, next, status);
    return;
  }
  const int blocks = Nh > 0 ? (Nh + CRF - 2) / (CRF - 1) : 1;
  k_cr_level<T><<<blocks, CRF, 0, s>>>(C, J, cur, level, next, status);
}

template <typename T>
void launch_cr_top(const DevChain &C, const DevJoints &J, const CRLevelT<T> &top, int level,
                   int *status, cudaStream_t s, double *out64, double *acc) {
  k_cr_top<T><<<1, 32, 0, s>>>(C, J, top, level, status, out64, acc);
}

template <typename T>
void launch_cr_back(const DevChain &C, const DevJoints &J, const CRLevelT<T> &cur, const CRLevelT<T> &next,
                    int level, cudaStream_t s, double *acc) {
  if (cur.N <= 0) return;
  if (cur.N / 2 <= CR_WARP_ROWS) {
    const int rows = (cur.N + 1) / 2;
    k_cr_back_w<T><<<(rows + 3) / 4, 128, 0, s>>>(cur, next, C, J, level, acc);
    return;
  }
  k_cr_back_pair<T><<<nblk((cur.N + 1) / 2, 128), 128, 0, s>>>(cur, next, C, J, level, acc);
}

template <typename T>
void launch_cr_rhs(const DevChain &C, const DevJoints &J, const CRLevelT<T> &cur, int level,
                   const CRLevelT<T> &next, cudaStream_t s) {
  if (next.N > 0) k_cr_rhs<T><<<nblk(next.N, 128), 128, 0, s>>>(C, J, cur, level, next);
}

template <typename T>
void launch_cr_tail(const DevChain &C, const DevJoints &J, const DevJoints &Jout, const CRLevelT<T> *d_lv,
                    int l0, int nl, bool rhs_only, T *cL, T *cR, T *Bn, int *status, double *acc,
                    cudaStream_t s) {
  k_cr_tail<T><<<1, cr_tail_threads<T>(), 0, s>>>(C, J, Jout, d_lv, l0, nl, rhs_only ? 1 : 0, cL, cR, Bn, status, acc);
}

#define MABD_CR_INSTANTIATE(T)                                                                       \
  template void launch_cr_level<T>(const DevChain &, const DevJoints &, const CRLevelT<T> &, int,     \
                                   const CRLevelT<T> &, int *, cudaStream_t);                       \
  template void launch_cr_top<T>(const DevChain &, const DevJoints &, const CRLevelT<T> &, int, int *, \
                                 cudaStream_t, double *, double *);                                 \
  template void launch_cr_back<T>(const DevChain &, const DevJoints &, const CRLevelT<T> &,           \
                                  const CRLevelT<T> &, int, cudaStream_t, double *);                \
  template void launch_cr_rhs<T>(const DevChain &, const DevJoints &, const CRLevelT<T> &, int,       \
                                 const CRLevelT<T> &, cudaStream_t);                               \
  template void launch_cr_tail<T>(const DevChain &, const DevJoints &, const DevJoints &,             \
                                  const CRLevelT<T> *, int, int, bool, T *, T *, T *, int *, double *, \
                                  cudaStream_t);
MABD_CR_INSTANTIATE(double)
MABD_CR_INSTANTIATE(float)
#undef MABD_CR_INSTANTIATE

void launch_mx_chain_gram(const DevBodies &B, const DevJoints &J, const DevIncidence &I,
                          const DevChain &C, cudaStream_t s, bool f32_blocks) {
  if (B.M <= 0) return;
  if (f32_blocks) k_mx_chain_gram<float><<<nblk(B.M, 128), 128, 0, s>>>(B, J, I, C);
  else k_mx_chain_gram<double><<<nblk(B.M, 128), 128, 0, s>>>(B, J, I, C);
}

}  // namespace mabd
