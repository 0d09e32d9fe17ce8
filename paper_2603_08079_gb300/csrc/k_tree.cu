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
// Everything of body j is kept in its rest frame (rows s [p;1] (x) R_j^T d),
// so a leaf uses the structured Hbar^{-1}; bodies with children factor their
// dense 12x12 Hhat (packed lower storage).  Variants for the bodies with
// children (one thread, or 8 or 4 lanes per body) and a persistent kernel
// (one CTA per tree) are chosen by the tuner in mabd_api.cpp.
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

template <typename S>
__device__ __forceinline__ void load_T16(const S *p, int M, int j, S h[16]) {
#pragma unroll
  for (int i = 0; i < 16; ++i) h[i] = __ldg(p + (size_t)i * M + j);
}

// a multiplier of the solve: to T.lam (FP64) and, when given, added to T.lam_acc
template <typename S>
__device__ __forceinline__ void put_lambda(const DevTreeT<S> &T, size_t o, S v) {
  const double v64 = to_f64(v);
  T.lam[o] = v64;
  if (T.lam_acc) T.lam_acc[o] += v64;
}

constexpr int RMAX = 10;  // rows eliminated at a root (two one-sided joints)
constexpr int TUP = 32;   // threads per block of the upward pass (one warp: small levels spread over SMs)

// Cholesky factor of a body's dense Hhat, kept in shared memory with the 78
// packed entries of a thread strided by the block size
template <typename S>
struct SmemL {
  S *base;
  __device__ __forceinline__ S &operator[](int e) const { return base[e * TUP]; }
};

template <typename S>
__device__ __forceinline__ bool chol12_smem(SmemL<S> A) {
  bool ok = true;
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    S s = A[p12(c, c)];
#pragma unroll
    for (int k = 0; k < c; ++k) {
      const S l = A[p12(c, k)];
      s -= l * l;
    }
    if (!(s > S(0))) {
      ok = false;
      s = S(1);
    }
    const S id = rsq(s);
    A[p12(c, c)] = id;  // reciprocal of the diagonal
#pragma unroll
    for (int r = c + 1; r < 12; ++r) {
      S t = A[p12(r, c)];
#pragma unroll
      for (int k = 0; k < c; ++k) t -= A[p12(r, k)] * A[p12(c, k)];
      A[p12(r, c)] = t * id;
    }
  }
  return ok;
}

template <typename S>
__device__ __noinline__ void chol12_solve_smem(SmemL<S> L, const S b[12], S x[12]) {
  S y[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    S s = b[i];
#pragma unroll
    for (int k = 0; k < i; ++k) s -= L[p12(i, k)] * y[k];
    y[i] = s * L[p12(i, i)];
  }
#pragma unroll
  for (int i = 11; i >= 0; --i) {
    S s = y[i];
#pragma unroll
    for (int k = i + 1; k < 12; ++k) s -= L[p12(k, i)] * x[k];
    x[i] = s * L[p12(i, i)];
  }
}

// dense Hbar written into the thread's shared-memory slots
template <typename S>
__device__ __forceinline__ void hbar_dense_smem(const DevBodies &B, int j, S ih2, SmemL<S> H) {
  const int M = B.M;
  const S s[3] = {ldgs<S>(B.sig + j), ldgs<S>(B.sig + M + j), ldgs<S>(B.sig + 2 * (size_t)M + j)};
  const S vm = ldgs<S>(B.vmu + j), vl = ldgs<S>(B.vlam + j), m = ldgs<S>(B.mass + j);
#pragma unroll
  for (int i = 0; i < 78; ++i) H[i] = S(0);
  const int dg[3] = {0, 4, 8};
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b <= a; ++b) H[p12(dg[a], dg[b])] = a == b ? s[a] * ih2 + S(2) * vm + vl : vl;
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

// Hbar x for the structured Hbar of body j (3x3 block of A's diagonal,
// transpose pairs, translation), from the body constants
template <typename S>
__device__ __forceinline__ void hbar_apply(const DevBodies &B, int j, S ih2, const S x[12],
                                           S y[12]) {
  const int M = B.M;
  const S s0 = ldgs<S>(B.sig + j), s1 = ldgs<S>(B.sig + M + j), s2 = ldgs<S>(B.sig + 2 * (size_t)M + j);
  const S vm = ldgs<S>(B.vmu + j), vl = ldgs<S>(B.vlam + j), m = ldgs<S>(B.mass + j);
  const S tr = vl * (x[0] + x[4] + x[8]);
  y[0] = (s0 * ih2 + S(2) * vm) * x[0] + tr;
  y[4] = (s1 * ih2 + S(2) * vm) * x[4] + tr;
  y[8] = (s2 * ih2 + S(2) * vm) * x[8] + tr;
  // pairs: (q1 = A(1,0), q3 = A(0,1)), (q2 = A(2,0), q6 = A(0,2)), (q5 = A(2,1), q7 = A(1,2))
  y[1] = (s0 * ih2 + vm) * x[1] + vm * x[3];
  y[3] = (s1 * ih2 + vm) * x[3] + vm * x[1];
  y[2] = (s0 * ih2 + vm) * x[2] + vm * x[6];
  y[6] = (s2 * ih2 + vm) * x[6] + vm * x[2];
  y[5] = (s1 * ih2 + vm) * x[5] + vm * x[7];
  y[7] = (s2 * ih2 + vm) * x[7] + vm * x[5];
  y[9] = m * ih2 * x[9];
  y[10] = m * ih2 * x[10];
  y[11] = m * ih2 * x[11];
}

// Upward pass for one body with N eliminated rows (its parent joint, or a
// root's one-sided joints when ROOT).
template <typename S, int N, bool ROOT>
__device__ __forceinline__ void up_body(const DevBodies &B, const DevJoints &J, const DevTreeT<S> &T, int j,
                                        const StepParams &p, int *status, SmemL<S> L) {
  const int M = B.M, K = J.K;
  S R[9];
  load_R(TB<S>::R(B), M, j, R);
  const int nch = T.ccount[j];
  S y[12];
  if (nch == 0) {
    load12(TB<S>::ubar(B), M, j, y);
  } else {
    // Hhat = Hbar + sum_children U U^T (dense, shared memory)
    const S ih2 = from_f64<S>(p.inv_h * p.inv_h);
    hbar_dense_smem(B, j, ih2, L);
    S ub[12], f[12];
    load12(TB<S>::ubar(B), M, j, ub);
    hbar_apply(B, j, ih2, ub, f);  // fbar = Hbar ubar
    const int c0 = T.cfirst[j];
    for (int c = c0; c < c0 + nch; ++c) {
#pragma unroll
      for (int a = 0; a < 12; ++a) f[a] -= T.v[(size_t)a * M + c];
      const int Cc = J.type[T.pjoint[c]] == 0 ? 3 : 5;
      for (int t = 0; t < Cc; ++t) {
        S u[12];
#pragma unroll
        for (int a = 0; a < 12; ++a) u[a] = T.U[(size_t)(5 * a + t) * M + c];
#pragma unroll
        for (int r = 0; r < 12; ++r)
#pragma unroll
          for (int cc = 0; cc <= r; ++cc) L[p12(r, cc)] += u[r] * u[cc];
      }
    }
    if (!chol12_smem(L)) set_status(status, ST_NOT_SPD);
    chol12_solve_smem(L, f, y);
  }
  // rows eliminated here (rest frame): s [p;1] (x) R^T d
  S E[N > 0 ? N : 1][3], P[4][3];
  int pt[N > 0 ? N : 1];
  int ks[2] = {-1, -1}, cs[2] = {0, 0};
  if constexpr (!ROOT) {
    ks[0] = T.pjoint[j];
    S E5[5][3], P2[2][3];
    int pt5[5];
    cs[0] = joint_rows_rest(J, ks[0], T.pside[j], R, E5, P2, pt5);
#pragma unroll
    for (int r = 0; r < N; ++r) {
      E[r][0] = E5[r][0]; E[r][1] = E5[r][1]; E[r][2] = E5[r][2];
      pt[r] = pt5[r];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      P[0][a] = P2[0][a];
      P[1][a] = P2[1][a];
    }
  } else {
    const int rid = T.root_id[j];
    int n = 0;
    for (int w = 0; w < 2; ++w) {
      const int k = T.root_joint[(size_t)w * T.nroots + rid];
      if (k < 0) continue;
      S E5[5][3], P2[2][3];
      int pt5[5];
      ks[w] = k;
      cs[w] = joint_rows_rest(J, k, T.root_side[(size_t)w * T.nroots + rid], R, E5, P2, pt5);
      for (int r = 0; r < cs[w] && n + r < (N > 0 ? N : 1); ++r) {
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
  S h[16];
  if (nch == 0) load_T16(TB<S>::hinv(B), M, j, h);
  // X_t = Hhat^{-1} w_t, D = G X, e = G y + C
  S D[N * (N + 1) / 2 > 0 ? N * (N + 1) / 2 : 1];
  S e[N > 0 ? N : 1];
  const S rr = from_f64<S>(T.crr);
  const int nr = T.nroots;
  const int rid = ROOT ? T.root_id[j] : -1;
#pragma unroll
  for (int t = 0; t < N; ++t) {
    S w[12], X[12];
    kron_row(P[pt[t]], E[t], w);
    if (nch == 0) hinv_apply(h, w, X);
    else chol12_solve_smem(L, w, X);
    S sy = S(0);
#pragma unroll
    for (int a = 0; a < 12; ++a) sy += w[a] * y[a];
    const int k = t < cs[0] ? ks[0] : ks[1];
    const int rl = t < cs[0] ? t : t - cs[0];
    e[t] = sy + rr * from_f64<S>(T.c[(size_t)rl * K + k]);
#pragma unroll
    for (int r = t; r < N; ++r) {
      S wr[12];
      kron_row(P[pt[r]], E[r], wr);
      S d = S(0);
#pragma unroll
      for (int a = 0; a < 12; ++a) d += wr[a] * X[a];
      D[p12(r, t)] = d;
    }
    if constexpr (!ROOT) {
#pragma unroll
      for (int a = 0; a < 12; ++a) T.X[(size_t)(5 * a + t) * M + j] = X[a];
    } else {
#pragma unroll
      for (int a = 0; a < 12; ++a) T.rX[(size_t)(RMAX * a + t) * nr + rid] = X[a];
    }
  }
  // Cholesky of D (reciprocal diagonal)
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
  if (!okd) set_status(status, ST_NOT_SPD);
  if constexpr (!ROOT) {
#pragma unroll
    for (int a = 0; a < 12; ++a) {
#pragma unroll
      for (int r = N; r < 5; ++r) T.X[(size_t)(5 * a + r) * M + j] = S(0);
      T.y[(size_t)a * M + j] = y[a];
    }
#pragma unroll
    for (int i = 0; i < 15; ++i) T.LD[(size_t)i * M + j] = i < N * (N + 1) / 2 ? D[i] : S(0);
#pragma unroll
    for (int r = 0; r < 5; ++r) T.e[(size_t)r * M + j] = r < N ? e[r] : S(0);
    // contribution to the parent (its rest frame): U = Pbar^T L_D^{-T}, v = U L_D^{-1} e
    const int par = T.parent[j];
    S Rp[9], Ep[5][3], Pp[2][3];
    int ptp[5];
    load_R(TB<S>::R(B), M, par, Rp);
    joint_rows_rest(J, ks[0], 1 - T.pside[j], Rp, Ep, Pp, ptp);
    S wl[N > 0 ? N : 1];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      S s = e[i];
#pragma unroll
      for (int k = 0; k < i; ++k) s -= D[p12(i, k)] * wl[k];
      wl[i] = s * D[p12(i, i)];
    }
#pragma unroll
    for (int blk = 0; blk < 4; ++blk)
#pragma unroll
      for (int a3 = 0; a3 < 3; ++a3) {
        const int a = 3 * blk + a3;
        S col[N > 0 ? N : 1], z[N > 0 ? N : 1];
#pragma unroll
        for (int r = 0; r < N; ++r) col[r] = (blk < 3 ? Pp[ptp[r]][blk] : S(1)) * Ep[r][a3];
        S vv = S(0);
#pragma unroll
        for (int i = 0; i < N; ++i) {
          S s = col[i];
#pragma unroll
          for (int k = 0; k < i; ++k) s -= D[p12(i, k)] * z[k];
          z[i] = s * D[p12(i, i)];
          T.U[(size_t)(5 * a + i) * M + j] = z[i];
          vv += z[i] * wl[i];
        }
#pragma unroll
        for (int i = N; i < 5; ++i) T.U[(size_t)(5 * a + i) * M + j] = S(0);
        T.v[(size_t)a * M + j] = vv;
      }
  } else {
#pragma unroll
    for (int a = 0; a < 12; ++a) {
#pragma unroll
      for (int r = N; r < RMAX; ++r) T.rX[(size_t)(RMAX * a + r) * nr + rid] = S(0);
      T.y[(size_t)a * M + j] = y[a];
    }
    for (int i = 0; i < RMAX * (RMAX + 1) / 2; ++i)
      T.rLD[(size_t)i * nr + rid] = i < N * (N + 1) / 2 ? D[i] : S(0);
    for (int r = 0; r < RMAX; ++r) T.re[(size_t)r * nr + rid] = r < N ? e[r] : S(0);
  }
}

// non-root bodies of a level: [lo, mid) have children (dense Hhat in shared
// memory), [mid, hi) are leaves (structured inverse)
template <typename S>
__global__ void __launch_bounds__(TUP) k_tree_up_inner(DevBodies B, DevJoints J, DevTreeT<S> T, int lo,
                                                       int hi, StepParams p, int *status) {
  __shared__ S sL[78 * TUP];
  const int i = lo + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= hi) return;
  const int j = T.order[i];
  if (T.parent[j] < 0) return;
  SmemL<S> L{sL + threadIdx.x};
  if (J.type[T.pjoint[j]] == 0) up_body<S, 3, false>(B, J, T, j, p, status, L);
  else up_body<S, 5, false>(B, J, T, j, p, status, L);
}

template <typename S>
__global__ void __launch_bounds__(128) k_tree_up_leaf(DevBodies B, DevJoints J, DevTreeT<S> T, int lo,
                                                      int hi, StepParams p, int *status) {
  const int i = lo + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= hi) return;
  const int j = T.order[i];
  if (T.parent[j] < 0) return;
  SmemL<S> L{nullptr};  // not touched: leaves have no children
  if (J.type[T.pjoint[j]] == 0) up_body<S, 3, false>(B, J, T, j, p, status, L);
  else up_body<S, 5, false>(B, J, T, j, p, status, L);
}

// ---------------------------------------------------------------------------
// lane-cooperative upward pass of the bodies with children
// ---------------------------------------------------------------------------
// The same elimination as up_body<S, N, false> for a body with children, done
// by a group of LANES lanes: the dense Hhat (78 packed entries), the rank
// updates of the children, the right-looking Cholesky's trailing updates and
// the Gram entries are dealt out over the lanes, and the lanes take the
// right-hand sides (f, then the N constraint rows) in turn.  A level with few such
// bodies then runs each body's dependent FP64 chain several times shorter.
constexpr int CG = 16;  // bodies (lane groups) per block

// entry (r, c), r >= c, of the packed lower triangle index e
__device__ __forceinline__ void unpack12(int e, int &r, int &c) {
  r = 0;
  while ((r + 1) * (r + 2) / 2 <= e) ++r;
  c = e - r * (r + 1) / 2;
}

// entry e of the dense Hbar (as hbar_dense)
template <typename S>
__device__ __forceinline__ S hbar_entry(int e, const S s[3], S vm, S vl, S m,
                                             S ih2) {
  int r, c;
  unpack12(e, r, c);
  const bool dr = (r == 0 || r == 4 || r == 8), dc = (c == 0 || c == 4 || c == 8);
  if (dr && dc) return r == c ? s[r / 4] * ih2 + S(2) * vm + vl : vl;
  if (r >= 9) return r == c ? m * ih2 : S(0);
  // transpose pairs (1,3), (2,6), (5,7); the first index has column ca, the second cb
  if (r == c) {
    switch (r) {
      case 1: case 2: return s[0] * ih2 + vm;
      case 3: case 5: return s[1] * ih2 + vm;
      case 6: case 7: return s[2] * ih2 + vm;
      default: return S(0);
    }
  }
  if ((r == 3 && c == 1) || (r == 6 && c == 2) || (r == 7 && c == 5)) return vm;
  return S(0);
}

template <typename S, int LANES, int N>
__device__ __forceinline__ void up_coop_body(const DevBodies &B, const DevJoints &J, const DevTreeT<S> &T, int j,
                                             const StepParams &p, int *status, int l, unsigned gmask,
                                             S *H, S (*Z)[6], S (*W)[5], S *Dg,
                                             S *Eg) {
  const int M = B.M, K = J.K;
  const S ih2 = from_f64<S>(p.inv_h * p.inv_h);
  // Hbar and f = Hbar ubar - sum_children v
  {
    const S s3[3] = {ldgs<S>(B.sig + j), ldgs<S>(B.sig + M + j), ldgs<S>(B.sig + 2 * (size_t)M + j)};
    const S vm = ldgs<S>(B.vmu + j), vl = ldgs<S>(B.vlam + j), m = ldgs<S>(B.mass + j);
    for (int e = l; e < 78; e += LANES) H[e] = hbar_entry(e, s3, vm, vl, m, ih2);
    S ub[12], hu[12];
    load12(TB<S>::ubar(B), M, j, ub);
    hbar_apply(B, j, ih2, ub, hu);
    const int c0 = T.cfirst[j], nch = T.ccount[j];
    for (int a = l; a < 12; a += LANES) {
      S f = S(0);
#pragma unroll
      for (int q = 0; q < 12; ++q)
        if (q == a) f = hu[q];
      for (int c = c0; c < c0 + nch; ++c) f -= T.v[(size_t)a * M + c];
      Z[a][0] = f;
    }
    __syncwarp(gmask);
    // Hhat = Hbar + sum_children U U^T (child's U staged in W)
    for (int c = c0; c < c0 + nch; ++c) {
      const int Cc = J.type[T.pjoint[c]] == 0 ? 3 : 5;
      for (int e = l; e < 12 * Cc; e += LANES) {
        const int a = e / Cc, t = e % Cc;
        W[a][t] = T.U[(size_t)(5 * a + t) * M + c];
      }
      __syncwarp(gmask);
      for (int e = l; e < 78; e += LANES) {
        int r, cc;
        unpack12(e, r, cc);
        S acc = S(0);
        for (int t = 0; t < Cc; ++t) acc += W[r][t] * W[cc][t];
        H[e] += acc;
      }
      __syncwarp(gmask);
    }
  }
  // Cholesky, right-looking, reciprocal diagonal in place
  bool ok = true;
  for (int c = 0; c < 12; ++c) {
    if (l == 0) {
      S d = H[p12(c, c)];
      if (!(d > S(0))) {
        ok = false;
        d = S(1);
      }
      H[p12(c, c)] = rsq(d);
    }
    __syncwarp(gmask);
    const S idc = H[p12(c, c)];
    for (int r = c + 1 + l; r < 12; r += LANES) H[p12(r, c)] *= idc;
    __syncwarp(gmask);
    int cnt = 0;
    for (int cc = c + 1; cc < 12; ++cc) {
      const S lcc = H[p12(cc, c)];
      for (int r = cc; r < 12; ++r, ++cnt)
        if (cnt % LANES == l) H[p12(r, cc)] -= H[p12(r, c)] * lcc;
    }
    __syncwarp(gmask);
  }
  if (!ok && l == 0) set_status(status, ST_NOT_SPD);
  // constraint rows of the parent joint on this body (rest frame), as
  // right-hand sides 1..N and kept in W
  const int kp = T.pjoint[j];
  {
    S R[9], E5[5][3], P2[2][3];
    int pt5[5];
    load_R(TB<S>::R(B), M, j, R);
    joint_rows_rest(J, kp, T.pside[j], R, E5, P2, pt5);
    for (int e = l; e < 12 * N; e += LANES) {
      const int a = e / N, t = e % N;
      const int blk = a / 3, a3 = a % 3;
      const S v = (blk < 3 ? P2[pt5[t]][blk] : S(1)) * E5[t][a3];
      W[a][t] = v;
      Z[a][1 + t] = v;
    }
  }
  __syncwarp(gmask);
  // lanes solve the columns in turn: y (column 0) and X_t = Hhat^{-1} w_t
  for (int col = l; col <= N; col += LANES) {
    S x[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      S v = Z[i][col];
#pragma unroll
      for (int k = 0; k < i; ++k) v -= H[p12(i, k)] * x[k];
      x[i] = v * H[p12(i, i)];
    }
#pragma unroll
    for (int i = 11; i >= 0; --i) {
      S v = x[i];
#pragma unroll
      for (int k = i + 1; k < 12; ++k) v -= H[p12(k, i)] * x[k];
      x[i] = v * H[p12(i, i)];
    }
#pragma unroll
    for (int i = 0; i < 12; ++i) Z[i][col] = x[i];
  }
  __syncwarp(gmask);
  // D_rt = w_r . X_t (packed), e_t = w_t . y + C
  constexpr int ND = N * (N + 1) / 2;
  const S rr = from_f64<S>(T.crr);
  for (int e = l; e < ND + N; e += LANES) {
    if (e < ND) {
      int r, t;
      unpack12(e, r, t);
      S d = S(0);
#pragma unroll
      for (int a = 0; a < 12; ++a) d += W[a][r] * Z[a][1 + t];
      Dg[e] = d;
    } else {
      const int t = e - ND;
      S d = S(0);
#pragma unroll
      for (int a = 0; a < 12; ++a) d += W[a][t] * Z[a][0];
      Eg[t] = d + rr * from_f64<S>(T.c[(size_t)t * K + kp]);
    }
  }
  // X and y out
  for (int e = l; e < 12 * 6; e += LANES) {
    const int a = e / 6, t = e % 6;
    if (t == 0) T.y[(size_t)a * M + j] = Z[a][0];
    else if (t <= 5) T.X[(size_t)(5 * a + t - 1) * M + j] = (t - 1 < N) ? Z[a][t] : S(0);
  }
  __syncwarp(gmask);
  // Cholesky of D (every lane), reciprocal diagonal
  S D[ND], ev[N];
#pragma unroll
  for (int i = 0; i < ND; ++i) D[i] = Dg[i];
#pragma unroll
  for (int i = 0; i < N; ++i) ev[i] = Eg[i];
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
  if (l == 0) {
#pragma unroll
    for (int i = 0; i < 15; ++i) T.LD[(size_t)i * M + j] = i < ND ? D[i] : S(0);
#pragma unroll
    for (int r = 0; r < 5; ++r) T.e[(size_t)r * M + j] = r < N ? ev[r] : S(0);
  }
  // contribution to the parent (its rest frame): U = Pbar^T L_D^{-T}, v = U L_D^{-1} e
  const int par = T.parent[j];
  S Rp[9], Ep[5][3], Pp[2][3];
  int ptp[5];
  load_R(TB<S>::R(B), M, par, Rp);
  joint_rows_rest(J, kp, 1 - T.pside[j], Rp, Ep, Pp, ptp);
  S wl[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    S s = ev[i];
#pragma unroll
    for (int k = 0; k < i; ++k) s -= D[p12(i, k)] * wl[k];
    wl[i] = s * D[p12(i, i)];
  }
  for (int a = l; a < 12; a += LANES) {
    const int blk = a / 3, a3 = a % 3;
    S col[N], z[N];
#pragma unroll
    for (int r = 0; r < N; ++r) col[r] = (blk < 3 ? Pp[ptp[r]][blk] : S(1)) * Ep[r][a3];
    S vv = S(0);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      S s = col[i];
#pragma unroll
      for (int k = 0; k < i; ++k) s -= D[p12(i, k)] * z[k];
      z[i] = s * D[p12(i, i)];
      T.U[(size_t)(5 * a + i) * M + j] = z[i];
      vv += z[i] * wl[i];
    }
#pragma unroll
    for (int i = N; i < 5; ++i) T.U[(size_t)(5 * a + i) * M + j] = S(0);
    T.v[(size_t)a * M + j] = vv;
  }
}

template <typename S, int LANES>
__global__ void __launch_bounds__(CG * LANES) k_tree_up_coop(DevBodies B, DevJoints J, DevTreeT<S> T, int lo,
                                                             int hi, StepParams p, int *status) {
  __shared__ S sH[CG][78];
  __shared__ S sZ[CG][12][6];
  __shared__ S sW[CG][12][5];
  __shared__ S sD[CG][15];
  __shared__ S sE[CG][5];
  const int g = threadIdx.x / LANES, l = threadIdx.x % LANES;
  const unsigned gmask = (LANES == 32) ? 0xffffffffu
                                       : (((1u << LANES) - 1u) << (((threadIdx.x & 31) / LANES) * LANES));
  const int i = lo + blockIdx.x * CG + g;
  if (i >= hi) return;  // uniform within the group
  const int j = T.order[i];
  if (T.parent[j] < 0) return;
  if (J.type[T.pjoint[j]] == 0)
    up_coop_body<S, LANES, 3>(B, J, T, j, p, status, l, gmask, sH[g], sZ[g], sW[g], sD[g], sE[g]);
  else
    up_coop_body<S, LANES, 5>(B, J, T, j, p, status, l, gmask, sH[g], sZ[g], sW[g], sD[g], sE[g]);
}

// each root variant compiled on its own (separate register allocation)
template <typename S, int N>
__device__ __noinline__ void up_root(const DevBodies &B, const DevJoints &J, const DevTreeT<S> &T, int j,
                                     const StepParams &p, int *status, SmemL<S> L) {
  up_body<S, N, true>(B, J, T, j, p, status, L);
}

// roots (level 0): their one-sided joints (0, 1 or 2 of 3 or 5 rows)
template <typename S>
__global__ void __launch_bounds__(TUP) k_tree_up_root(DevBodies B, DevJoints J, DevTreeT<S> T, int lo,
                                                      int hi, StepParams p, int *status) {
  __shared__ S sL[78 * TUP];
  const int j = lo + blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= hi || T.parent[j] >= 0) return;
  SmemL<S> L{sL + threadIdx.x};
  const int rid = T.root_id[j];
  int n = 0;
  for (int w = 0; w < 2; ++w) {
    const int k = T.root_joint[(size_t)w * T.nroots + rid];
    if (k >= 0) n += J.type[k] == 0 ? 3 : 5;
  }
  switch (n) {
    case 0: up_root<S, 0>(B, J, T, j, p, status, L); break;
    case 3: up_root<S, 3>(B, J, T, j, p, status, L); break;
    case 5: up_root<S, 5>(B, J, T, j, p, status, L); break;
    case 6: up_root<S, 6>(B, J, T, j, p, status, L); break;
    case 8: up_root<S, 8>(B, J, T, j, p, status, L); break;
    default: up_root<S, 10>(B, J, T, j, p, status, L); break;
  }
}

// downward pass of a non-root body with N rows in its parent joint
template <typename S, int N>
__device__ __forceinline__ void down_body(const DevBodies &B, const DevJoints &J, const DevTreeT<S> &T,
                                          int j, int par, S dqb[12]) {
  const int M = B.M, K = J.K;
  const int k = T.pjoint[j];
  constexpr int type = N == 3 ? 0 : 1;
  const int pside = 1 - T.pside[j];
  // P dq_parent: rows s_p d_r^T J(p_r) dq_p in the world frame
  S dqp[12];
  load12(T.dq, M, par, dqp);
  S pts[2][3];
  load3(JP<S>::p1(J, pside), K, k, pts[0]);
  if (type == 1) load3(JP<S>::p2(J, pside), K, k, pts[1]);
  S x[2][3];
#pragma unroll
  for (int q = 0; q < 1 + type; ++q)
#pragma unroll
    for (int a = 0; a < 3; ++a)
      x[q][a] = dqp[a] * pts[q][0] + dqp[3 + a] * pts[q][1] + dqp[6 + a] * pts[q][2] + dqp[9 + a];
  S RH[9];
  if (type == 1) load_R(JP<S>::RH(J), K, k, RH);
  const S sp = pside == 0 ? S(1) : -S(1);
  S rhs[N], t[N], lam[N], LD[N * (N + 1) / 2];
#pragma unroll
  for (int r = 0; r < N; ++r) {
    S d[3];
    row_dir(type, RH, r, d);
    const int q = r < 3 ? 0 : 1;
    rhs[r] = T.e[(size_t)r * M + j] + sp * (d[0] * x[q][0] + d[1] * x[q][1] + d[2] * x[q][2]);
  }
#pragma unroll
  for (int i = 0; i < N * (N + 1) / 2; ++i) LD[i] = T.LD[(size_t)i * M + j];
  // L_D stores reciprocal diagonals
#pragma unroll
  for (int i = 0; i < N; ++i) {
    S s = rhs[i];
#pragma unroll
    for (int q = 0; q < i; ++q) s -= LD[p12(i, q)] * t[q];
    t[i] = s * LD[p12(i, i)];
  }
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    S s = t[i];
#pragma unroll
    for (int q = i + 1; q < N; ++q) s -= LD[p12(q, i)] * lam[q];
    lam[i] = s * LD[p12(i, i)];
  }
#pragma unroll
  for (int r = 0; r < N; ++r) put_lambda(T, (size_t)r * K + k, lam[r]);
#pragma unroll
  for (int a = 0; a < 12; ++a) {
    S s = T.y[(size_t)a * M + j];
#pragma unroll
    for (int r = 0; r < N; ++r) s -= T.X[(size_t)(5 * a + r) * M + j] * lam[r];
    dqb[a] = s;
  }
}

// downward pass of body j: lambda of its parent joint (or of a root's
// one-sided joints), dq, and the state update
template <typename S>
__device__ __forceinline__ void tree_down_one(const DevBodies &B, const DevJoints &J, const DevTreeT<S> &T,
                                              int j, const StepParams &p) {
  const int M = B.M, K = J.K;
  const int par = T.parent[j];
  S dqb[12];
  if (par >= 0) {
    if (J.type[T.pjoint[j]] == 0) down_body<S, 3>(B, J, T, j, par, dqb);
    else down_body<S, 5>(B, J, T, j, par, dqb);
  } else {
    const int rid = T.root_id[j];
    const int nr = T.nroots;
    int n = 0, cs[2] = {0, 0}, ks[2] = {-1, -1};
    for (int w = 0; w < 2; ++w) {
      ks[w] = rid >= 0 ? T.root_joint[(size_t)w * nr + rid] : -1;
      cs[w] = ks[w] < 0 ? 0 : (J.type[ks[w]] == 0 ? 3 : 5);
      n += cs[w];
    }
    S lam[RMAX], t[RMAX], e[RMAX], LD[RMAX * (RMAX + 1) / 2];
    for (int r = 0; r < n; ++r) e[r] = T.re[(size_t)r * nr + rid];
    for (int i = 0; i < n * (n + 1) / 2; ++i) LD[i] = T.rLD[(size_t)i * nr + rid];
    for (int i = 0; i < n; ++i) {  // reciprocal diagonals
      S s = e[i];
      for (int q = 0; q < i; ++q) s -= LD[p12(i, q)] * t[q];
      t[i] = s * LD[p12(i, i)];
    }
    for (int i = n - 1; i >= 0; --i) {
      S s = t[i];
      for (int q = i + 1; q < n; ++q) s -= LD[p12(q, i)] * lam[q];
      lam[i] = s * LD[p12(i, i)];
    }
    for (int r = 0; r < n; ++r) {
      const int w = r < cs[0] ? 0 : 1;
      put_lambda(T, (size_t)(r - (w ? cs[0] : 0)) * K + ks[w], lam[r]);
    }
    for (int a = 0; a < 12; ++a) {
      S s = T.y[(size_t)a * M + j];
      for (int r = 0; r < n; ++r) s -= T.rX[(size_t)(RMAX * a + r) * nr + rid] * lam[r];
      dqb[a] = s;
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

template <typename S>
__global__ void __launch_bounds__(128) k_tree_down(DevBodies B, DevJoints J, DevTreeT<S> T, int lo,
                                                   int hi, StepParams p) {
  const int j = lo + blockIdx.x * blockDim.x + threadIdx.x;
  if (j < hi) tree_down_one(B, J, T, j, p);
}

// ---------------------------------------------------------------------------
// persistent forest kernel: one block per tree, both passes
// ---------------------------------------------------------------------------
constexpr int FT = 128;  // threads per block

template <typename S, int LANES>
constexpr size_t forest_smem() {
  return sizeof(S) * (78 * TUP + (FT / LANES) * (78 + 12 * 6 + 12 * 5 + 15 + 5));
}

// each per-body path compiled on its own (separate register allocation)
template <typename S, int LANES, int N>
__device__ __noinline__ void coop_one(const DevBodies &B, const DevJoints &J, const DevTreeT<S> &T, int j,
                                      const StepParams &p, int *status, int l, unsigned gmask, S *H,
                                      S (*Z)[6], S (*W)[5], S *Dg, S *Eg) {
  up_coop_body<S, LANES, N>(B, J, T, j, p, status, l, gmask, H, Z, W, Dg, Eg);
}

template <typename S, int N>
__device__ __noinline__ void leaf_one(const DevBodies &B, const DevJoints &J, const DevTreeT<S> &T, int j,
                                      const StepParams &p, int *status) {
  SmemL<S> L{nullptr};
  up_body<S, N, false>(B, J, T, j, p, status, L);
}

template <typename S>
__device__ __noinline__ void down_one(const DevBodies &B, const DevJoints &J, const DevTreeT<S> &T, int j,
                                      const StepParams &p) {
  tree_down_one(B, J, T, j, p);
}

template <typename S, int N>
__device__ __noinline__ void inner_one(const DevBodies &B, const DevJoints &J, const DevTreeT<S> &T, int j,
                                       const StepParams &p, int *status, SmemL<S> L) {
  up_body<S, N, false>(B, J, T, j, p, status, L);
}

template <typename S, int LANES>
__global__ void __launch_bounds__(FT) k_tree_forest(DevBodies B, DevJoints J, DevTreeT<S> T, DevForest F,
                                                    StepParams p, int *status) {
  extern __shared__ __align__(16) unsigned char forest_raw[];
  S *smem = reinterpret_cast<S *>(forest_raw);
  constexpr int NG = FT / LANES;
  S *sL = smem;                       // root's dense factor, stride TUP
  S *gbase = smem + 78 * TUP;
  const int g = threadIdx.x / LANES, l = threadIdx.x % LANES;
  const unsigned gmask = (((1u << LANES) - 1u) << (((threadIdx.x & 31) / LANES) * LANES));
  S *H = gbase + (size_t)g * (78 + 72 + 60 + 15 + 5);
  S(*Z)[6] = reinterpret_cast<S(*)[6]>(H + 78);
  S(*W)[5] = reinterpret_cast<S(*)[5]>(H + 78 + 72);
  S *Dg = H + 78 + 72 + 60, *Eg = Dg + 15;
  for (int t = blockIdx.x; t < F.ntrees; t += gridDim.x) {
    const int r0 = F.tlvl[t], nl = F.tnl[t];
    // upward, deepest level first
    for (int d = nl - 1; d >= 1; --d) {
      const int lo = F.lo[r0 + d], mid = F.mid[r0 + d], hi = F.lo[r0 + d + 1];
      for (int i = lo + g; i < mid; i += NG) {
        const int j = F.order[i];
        if (J.type[T.pjoint[j]] == 0) coop_one<S, LANES, 3>(B, J, T, j, p, status, l, gmask, H, Z, W, Dg, Eg);
        else coop_one<S, LANES, 5>(B, J, T, j, p, status, l, gmask, H, Z, W, Dg, Eg);
      }
      for (int i = mid + threadIdx.x; i < hi; i += FT) {
        const int j = F.order[i];
        if (J.type[T.pjoint[j]] == 0) leaf_one<S, 3>(B, J, T, j, p, status);
        else leaf_one<S, 5>(B, J, T, j, p, status);
      }
      __syncthreads();
    }
    // the root
    if (threadIdx.x == 0) {
      const int j = F.order[F.lo[r0]];
      const int rid = T.root_id[j];
      int n = 0;
      for (int w = 0; w < 2; ++w) {
        const int k = T.root_joint[(size_t)w * T.nroots + rid];
        if (k >= 0) n += J.type[k] == 0 ? 3 : 5;
      }
      SmemL<S> L{sL};
      switch (n) {
        case 0: up_root<S, 0>(B, J, T, j, p, status, L); break;
        case 3: up_root<S, 3>(B, J, T, j, p, status, L); break;
        case 5: up_root<S, 5>(B, J, T, j, p, status, L); break;
        case 6: up_root<S, 6>(B, J, T, j, p, status, L); break;
        case 8: up_root<S, 8>(B, J, T, j, p, status, L); break;
        default: up_root<S, 10>(B, J, T, j, p, status, L); break;
      }
    }
    __syncthreads();
    // downward, root first
    for (int d = 0; d < nl; ++d) {
      const int lo = F.lo[r0 + d], hi = F.lo[r0 + d + 1];
      for (int i = lo + threadIdx.x; i < hi; i += FT) down_one(B, J, T, F.order[i], p);
      __syncthreads();
    }
  }
}

template <typename S>
void launch_tree_forest(const DevBodies &B, const DevJoints &J, const DevTreeT<S> &T, const DevForest &F,
                        const StepParams &p, int *status, cudaStream_t s, int lanes) {
  if (F.ntrees <= 0) return;
  if (lanes == 4) {
    constexpr size_t sm = forest_smem<S, 4>();
    static bool set = false;
    if (!set) {
      cudaFuncSetAttribute(k_tree_forest<S, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      set = true;
    }
    k_tree_forest<S, 4><<<F.ntrees, FT, sm, s>>>(B, J, T, F, p, status);
  } else {
    constexpr size_t sm = forest_smem<S, 8>();
    static bool set = false;
    if (!set) {
      cudaFuncSetAttribute(k_tree_forest<S, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      set = true;
    }
    k_tree_forest<S, 8><<<F.ntrees, FT, sm, s>>>(B, J, T, F, p, status);
  }
}

// One tree level in one launch: blocks [0, nbi) eliminate the bodies with
// children (one per thread, TUP threads per block, or LANES lanes per body),
// the other blocks the leaves (one per thread); the two sets do not depend on
// each other, so their latencies overlap instead of adding up.
template <typename S, int LANES>
__global__ void __launch_bounds__(LANES == 0 ? TUP : CG * LANES)
    k_tree_up_level(DevBodies B, DevJoints J, DevTreeT<S> T, int lo, int mid, int hi, int nbi, StepParams p,
                    int *status) {
  if ((int)blockIdx.x >= nbi) {
    const int i = mid + ((int)blockIdx.x - nbi) * blockDim.x + threadIdx.x;
    if (i >= hi) return;
    const int j = T.order[i];
    if (T.parent[j] < 0) return;
    if (J.type[T.pjoint[j]] == 0) leaf_one<S, 3>(B, J, T, j, p, status);
    else leaf_one<S, 5>(B, J, T, j, p, status);
    return;
  }
  if constexpr (LANES == 0) {
    __shared__ S sL[78 * TUP];
    const int i = lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= mid) return;
    const int j = T.order[i];
    if (T.parent[j] < 0) return;
    SmemL<S> L{sL + threadIdx.x};
    if (J.type[T.pjoint[j]] == 0) inner_one<S, 3>(B, J, T, j, p, status, L);
    else inner_one<S, 5>(B, J, T, j, p, status, L);
  } else {
    __shared__ S sH[CG][78];
    __shared__ S sZ[CG][12][6];
    __shared__ S sW[CG][12][5];
    __shared__ S sD[CG][15];
    __shared__ S sE[CG][5];
    const int g = threadIdx.x / LANES, l = threadIdx.x % LANES;
    const unsigned gmask = (((1u << LANES) - 1u) << (((threadIdx.x & 31) / LANES) * LANES));
    const int i = lo + blockIdx.x * CG + g;
    if (i >= mid) return;
    const int j = T.order[i];
    if (T.parent[j] < 0) return;
    if (J.type[T.pjoint[j]] == 0)
      coop_one<S, LANES, 3>(B, J, T, j, p, status, l, gmask, sH[g], sZ[g], sW[g], sD[g], sE[g]);
    else
      coop_one<S, LANES, 5>(B, J, T, j, p, status, l, gmask, sH[g], sZ[g], sW[g], sD[g], sE[g]);
  }
}

template <typename S>
void launch_tree_up(const DevBodies &B, const DevJoints &J, const DevTreeT<S> &T, int lo, int mid,
                    int hi, bool roots, const StepParams &p, int *status, cudaStream_t s, int variant) {
  if (!roots && mid > lo && hi > mid) {
    const int ni = mid - lo, nl = hi - mid;
    if (variant == TREE_UP_COOP8) {
      const int nbi = (ni + CG - 1) / CG, nbl = (nl + CG * 8 - 1) / (CG * 8);
      k_tree_up_level<S, 8><<<nbi + nbl, CG * 8, 0, s>>>(B, J, T, lo, mid, hi, nbi, p, status);
    } else if (variant == TREE_UP_COOP4) {
      const int nbi = (ni + CG - 1) / CG, nbl = (nl + CG * 4 - 1) / (CG * 4);
      k_tree_up_level<S, 4><<<nbi + nbl, CG * 4, 0, s>>>(B, J, T, lo, mid, hi, nbi, p, status);
    } else {
      const int nbi = (ni + TUP - 1) / TUP, nbl = (nl + TUP - 1) / TUP;
      k_tree_up_level<S, 0><<<nbi + nbl, TUP, 0, s>>>(B, J, T, lo, mid, hi, nbi, p, status);
    }
    return;
  }
  if (roots) {
    if (hi > lo) k_tree_up_root<S><<<(hi - lo + TUP - 1) / TUP, TUP, 0, s>>>(B, J, T, lo, hi, p, status);
    return;
  }
  if (mid > lo) {
    const int n = mid - lo;
    if (variant == TREE_UP_COOP8)
      k_tree_up_coop<S, 8><<<(n + CG - 1) / CG, CG * 8, 0, s>>>(B, J, T, lo, mid, p, status);
    else if (variant == TREE_UP_COOP4)
      k_tree_up_coop<S, 4><<<(n + CG - 1) / CG, CG * 4, 0, s>>>(B, J, T, lo, mid, p, status);
    else
      k_tree_up_inner<S><<<(n + TUP - 1) / TUP, TUP, 0, s>>>(B, J, T, lo, mid, p, status);
  }
  if (hi > mid) k_tree_up_leaf<S><<<(hi - mid + 127) / 128, 128, 0, s>>>(B, J, T, mid, hi, p, status);
}

template <typename S>
void launch_tree_down(const DevBodies &B, const DevJoints &J, const DevTreeT<S> &T, int lo, int hi,
                      const StepParams &p, int * /*status*/, cudaStream_t s) {
  const int n = hi - lo;
  if (n > 0) k_tree_down<S><<<(n + 127) / 128, 128, 0, s>>>(B, J, T, lo, hi, p);
}

#define MABD_TREE_INSTANTIATE(S)                                                                   \
  template void launch_tree_forest<S>(const DevBodies &, const DevJoints &, const DevTreeT<S> &,    \
                                      const DevForest &, const StepParams &, int *, cudaStream_t,  \
                                      int);                                                        \
  template void launch_tree_up<S>(const DevBodies &, const DevJoints &, const DevTreeT<S> &, int,   \
                                  int, int, bool, const StepParams &, int *, cudaStream_t, int);   \
  template void launch_tree_down<S>(const DevBodies &, const DevJoints &, const DevTreeT<S> &, int, \
                                    int, const StepParams &, int *, cudaStream_t);
MABD_TREE_INSTANTIATE(double)
MABD_TREE_INSTANTIATE(float)
#undef MABD_TREE_INSTANTIATE

}  // namespace mabd
