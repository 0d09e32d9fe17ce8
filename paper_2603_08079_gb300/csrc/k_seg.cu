// Segment-tiled chain step of the mixed-precision form (FP32 products and
// FP32 block cyclic reduction, refined by one FP64-level correction sweep).
//
// The chain's dual (Eq. chain-btd, Sec. 5.2) is block tridiagonal over the
// joints in path order: joint k joins path bodies k - 1 + sigma and
// k + sigma, and two neighbouring joints couple through the body they share
// (Eq. chain-Schur-blocks).  The rows are cut into tiles of SEG_T joints.  One
// CTA per tile
//   - reads the states of the tile's SEG_T + 2 bodies (its own SEG_T and one
//     halo body at each end) and its joints, forms the polar rotations
//     (Eq. polar), the rest-frame rhs and u = Hbar^{-1} f (Eq. abd_final), the
//     constraint values, the joint frames and b = G u + C (Eq. ball, hinge,
//     pcpq), and the Gram blocks of each body (Eq. chain-Schur-blocks), all
//     into shared memory;
//   - eliminates rows 1 .. SEG_T - 1 of the tile by block cyclic reduction in
//     shared memory: at level l the rows s (2m + 1), s = 2^l, are eliminated
//     into their neighbours s 2m and s (2m + 2); row SEG_T is the next tile's
//     first row, which receives (accumulated in the tile) what the tile's
//     eliminations add to it;
//   - writes only its first row's reduced block, its coupling to the next
//     tile's first row, and those accumulated updates.
// The first rows of all tiles form a block-tridiagonal system of
// ceil(K / SEG_T) rows, reduced by tiles of SEG_UP_T rows the same way until a
// single CTA solves it; back-substitution runs down the same levels.
//
// One step, with one correction sweep (the refinement of the mixed form):
//   FIRST  the approximate solve: per-body and per-joint work, Gram blocks,
//          factorization and forward elimination of b (y of every eliminated
//          row kept in ytile);
//   CORR   back-substitution of the approximate multipliers lambda0, then per
//          body dq0 = u - Hbar^{-1} g(lambda0), the primal residual
//          r_p = fbar - Hbar dq0 - g(lambda0) in double-float and
//          z = Hbar^{-1} r_p; per joint the dual residual r_d = C + G dq0 in
//          double-float and the correction's rhs G z + r_d, forward-eliminated
//          through the tile's factors (recomputed from the same data);
//   FINAL  back-substitution of the correction dlambda; lambda = lambda0 +
//          dlambda; dq = dq0 + z - Hbar^{-1} g(dlambda); q += diag4(R) dq,
//          qdot = diag4(R) dq / h (implicit Euler, Sec. 3.4).
// Each pass recomputes the Gram blocks and the tile's factorization from the
// rotations written by FIRST instead of storing factors: the data they are
// built from is read by the pass anyway.
//
// All blocks are kept 5x5 (a ball joint's two extra rows carry an identity
// diagonal and decouple exactly).  Packed lower-triangular 5x5 storage:
// entry (r, c), r >= c, at r (r + 1) / 2 + c; couplings row-major.
#include "mabd_mx.cuh"

namespace mabd {

constexpr int SEG_NT = SEG_T;      // one thread per tile body and tile row (threads 0, 1 take the halo)
constexpr int SEG_MINB = 384 / SEG_T;  // resident tiles per SM the register budget is set for
constexpr int SEG_NB = SEG_T + 2;   // tile bodies: halo 0, own 1 .. SEG_T, halo SEG_T + 1
constexpr int SEG_NR = SEG_T + 4;   // tile rows: SEG_T joints and the next tile's first row (padded to 4)
constexpr int UP_NT = 128;
// a tile's factor block: D, Bm, Ya of every tile row (65 x SEG_NR floats)
constexpr int SEG_FAC = 65 * SEG_NR;
static_assert(SEG_FAC % 4 == 0, "factor block of whole 16-byte words");
constexpr int UP_NR = SEG_UP_T + 4;

__host__ __device__ constexpr int pk5(int r, int c) { return r >= c ? r * (r + 1) / 2 + c : c * (c + 1) / 2 + r; }

// ---------------------------------------------------------------------------
// block cyclic reduction of a tile held in shared memory (rows 0 .. T, row T
// external).  Component c of row r of an array X lives at X[c * NR + r].
// ---------------------------------------------------------------------------
struct TileV {
  float *D;   // [15]: the row's block; an eliminated row's Cholesky factor L (reciprocal diagonal)
  float *Bm;  // [25]: coupling to the right neighbour of the current level; Yb of an eliminated row
  float *Ya;  // [25]: Ya of an eliminated row
  float *b;   // [5]: rhs; y of an eliminated row; multipliers after back-substitution
};

__device__ __forceinline__ void chol5(float L[15], int *status) {
  bool ok = true;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    float sum = L[pk5(c, c)];
#pragma unroll
    for (int k = 0; k < c; ++k) sum -= L[pk5(c, k)] * L[pk5(c, k)];
    if (!(sum > 0.f)) {
      ok = false;
      sum = 1.f;
    }
    const float id = rsqrtf(sum);
    L[pk5(c, c)] = id;
#pragma unroll
    for (int r = c + 1; r < 5; ++r) {
      float t = L[pk5(r, c)];
#pragma unroll
      for (int k = 0; k < c; ++k) t -= L[pk5(r, k)] * L[pk5(c, k)];
      L[pk5(r, c)] = t * id;
    }
  }
  if (!ok) set_status(status, ST_NOT_SPD);
}

// x = L^{-1} v
__device__ __forceinline__ void fwd5(const float L[15], const float v[5], float x[5]) {
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    float t = v[i];
#pragma unroll
    for (int k = 0; k < i; ++k) t -= L[pk5(i, k)] * x[k];
    x[i] = t * L[pk5(i, i)];
  }
}

// x = L^{-T} v
__device__ __forceinline__ void bwd5(const float L[15], const float v[5], float x[5]) {
#pragma unroll
  for (int i = 4; i >= 0; --i) {
    float t = v[i];
#pragma unroll
    for (int k = i + 1; k < 5; ++k) t -= L[pk5(k, i)] * x[k];
    x[i] = t * L[pk5(i, i)];
  }
}

// Eliminate row r (left neighbour r - s, right neighbour r + s): factor its
// block, store L, Ya = L^{-1} B_left^T, Yb = L^{-1} B_r and y = L^{-1} b_r,
// apply the Schur update to the left neighbour (block, rhs, and its coupling,
// which now reaches the right neighbour: -Ya^T Yb) and return the right
// neighbour's update (Yb^T Yb, Yb^T y).
template <int NR>
__device__ __forceinline__ void elim_row(const TileV &V, int r, int s, bool rhs, float dD[15], float db[5],
                                         int *status) {
  const int lft = r - s;
  float L[15];
#pragma unroll
  for (int i = 0; i < 15; ++i) L[i] = V.D[i * NR + r];
  chol5(L, status);
#pragma unroll
  for (int i = 0; i < 15; ++i) V.D[i * NR + r] = L[i];
  float y[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  if (rhs) {
    float v[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) v[i] = V.b[i * NR + r];
    fwd5(L, v, y);
#pragma unroll
    for (int i = 0; i < 5; ++i) V.b[i * NR + r] = y[i];
  }
  float Ya[25], Yb[25];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    float v[5], x[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) v[i] = V.Bm[(5 * i + c) * NR + r];
    fwd5(L, v, x);
#pragma unroll
    for (int i = 0; i < 5; ++i) Yb[5 * i + c] = x[i];
#pragma unroll
    for (int i = 0; i < 5; ++i) v[i] = V.Bm[(5 * c + i) * NR + lft];
    fwd5(L, v, x);
#pragma unroll
    for (int i = 0; i < 5; ++i) Ya[5 * i + c] = x[i];
  }
#pragma unroll
  for (int i = 0; i < 25; ++i) {
    V.Bm[i * NR + r] = Yb[i];
    V.Ya[i * NR + r] = Ya[i];
  }
  // left neighbour: D -= Ya^T Ya, b -= Ya^T y, coupling to the right neighbour -Ya^T Yb
#pragma unroll
  for (int p = 0; p < 5; ++p) {
#pragma unroll
    for (int q = 0; q <= p; ++q) {
      float t = 0.f;
#pragma unroll
      for (int i = 0; i < 5; ++i) t += Ya[5 * i + p] * Ya[5 * i + q];
      V.D[pk5(p, q) * NR + lft] -= t;
    }
    if (rhs) {
      float t = 0.f;
#pragma unroll
      for (int i = 0; i < 5; ++i) t += Ya[5 * i + p] * y[i];
      V.b[p * NR + lft] -= t;
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      float t = 0.f;
#pragma unroll
      for (int i = 0; i < 5; ++i) t += Ya[5 * i + p] * Yb[5 * i + c];
      V.Bm[(5 * p + c) * NR + lft] = -t;
    }
  }
  // right neighbour's update, applied by the caller after a barrier
#pragma unroll
  for (int p = 0; p < 5; ++p) {
#pragma unroll
    for (int q = 0; q <= p; ++q) {
      float t = 0.f;
#pragma unroll
      for (int i = 0; i < 5; ++i) t += Yb[5 * i + p] * Yb[5 * i + q];
      dD[pk5(p, q)] = t;
    }
    float t = 0.f;
#pragma unroll
    for (int i = 0; i < 5; ++i) t += Yb[5 * i + p] * y[i];
    db[p] = t;
  }
}

// Eliminate row r as elim_row does, with a group of G = 16 or 32 lanes of a
// warp (gl the lane's index in the group, gbase its first lane, gmask the
// group's lanes): every lane factors the block; lane c < 11 solves column c
// (0-4: Ya = L^{-1} B_left^T, 5-9: Yb = L^{-1} B_r, 10: y) and stores it; the
// entries of the neighbours' updates are dealt out over the lanes, each a dot
// product of two columns fetched from their lanes by shuffles.  The left
// neighbour's 45 entries (D -= Ya^T Ya, b -= Ya^T y, coupling -Ya^T Yb) are
// applied at once, the right neighbour's 20 (Yb^T Yb, Yb^T y) kept in Rt[20]
// of row r until the caller's barrier.  Entry tables: packed lower 5x5
// position e -> (p, q).
__device__ __constant__ int8_t kPkP[15] = {0, 1, 1, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4, 4};
__device__ __constant__ int8_t kPkQ[15] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3, 0, 1, 2, 3, 4};

template <int NR>
__device__ __forceinline__ void elim_row_grp(const TileV &V, float *Rt, int r, int s, bool rhs, int G, int gl,
                                             int gbase, unsigned gmask, int *status) {
  const int lft = r - s;
  float L[15];
#pragma unroll
  for (int i = 0; i < 15; ++i) L[i] = V.D[i * NR + r];
  chol5(L, gl == 0 ? status : nullptr);
  // this lane's column (gl < 11)
  float col[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  if (gl < (rhs ? 11 : 10)) {
    float v[5];
    if (gl < 5) {
#pragma unroll
      for (int i = 0; i < 5; ++i) v[i] = V.Bm[(5 * gl + i) * NR + lft];
    } else if (gl < 10) {
#pragma unroll
      for (int i = 0; i < 5; ++i) v[i] = V.Bm[(5 * i + gl - 5) * NR + r];
    } else {
#pragma unroll
      for (int i = 0; i < 5; ++i) v[i] = V.b[i * NR + r];
    }
    fwd5(L, v, col);
  }
  __syncwarp(gmask);  // every lane has read D, B_left, B_r and b of row r
  if (gl == 0)
#pragma unroll
    for (int i = 0; i < 15; ++i) V.D[i * NR + r] = L[i];
  if (gl < 5) {
#pragma unroll
    for (int i = 0; i < 5; ++i) V.Ya[(5 * i + gl) * NR + r] = col[i];
  } else if (gl < 10) {
#pragma unroll
    for (int i = 0; i < 5; ++i) V.Bm[(5 * i + gl - 5) * NR + r] = col[i];
  } else if (gl == 10 && rhs) {
#pragma unroll
    for (int i = 0; i < 5; ++i) V.b[i * NR + r] = col[i];
  }
  // entries: 0-14 D_left, 15-19 b_left, 20-44 coupling, 45-59 D_right, 60-64 b_right
  for (int e0 = 0; e0 < 65; e0 += G) {
    const int e = e0 + gl;
    int ca = 0, cb = 0;  // the two columns of the entry
    if (e < 15) {
      ca = kPkP[e];
      cb = kPkQ[e];
    } else if (e < 20) {
      ca = e - 15;
      cb = 10;
    } else if (e < 45) {
      ca = (e - 20) / 5;
      cb = 5 + (e - 20) % 5;
    } else if (e < 60) {
      ca = 5 + kPkP[e - 45];
      cb = 5 + kPkQ[e - 45];
    } else if (e < 65) {
      ca = 5 + e - 60;
      cb = 10;
    }
    float t = 0.f;
#pragma unroll
    for (int i = 0; i < 5; ++i) t += __shfl_sync(gmask, col[i], gbase + ca) * __shfl_sync(gmask, col[i], gbase + cb);
    if (e < 15) V.D[e * NR + lft] -= t;
    else if (e < 20) {
      if (rhs) V.b[(e - 15) * NR + lft] -= t;
    } else if (e < 45) V.Bm[(e - 20) * NR + lft] = -t;
    else if (e < 65) Rt[(e - 45) * NR + r] = (e < 60 || rhs) ? t : 0.f;
  }
}

// factorization of rows 1 .. T - 1 (and forward elimination of b when rhs),
// all levels (T a power of two, T / 2 <= NT); every thread of the block
// calls it.  Levels with at least NT / 16 eliminations run one thread per row
// (the register form); smaller levels a group of G = NT / nel lanes (16 or
// 32) per row.  Rt: scratch of 20 values per row for the group form.
template <int NR, int NT>
__device__ __forceinline__ void tile_factor(const TileV &V, float *Rt, int T, bool rhs, int *status) {
  const int tid = threadIdx.x;
#pragma unroll 1
  for (int s = 1; s < T; s <<= 1) {
    const int nel = T / (2 * s);
    if (nel * 16 > NT) {
      float dD[15], db[5];
      int r = -1;
      if (tid < nel) {
        r = s * (2 * tid + 1);
        elim_row<NR>(V, r, s, rhs, dD, db, status);
      }
      __syncthreads();
      if (r >= 0) {
        const int rr = r + s;
#pragma unroll
        for (int i = 0; i < 15; ++i) V.D[i * NR + rr] -= dD[i];
        if (rhs)
#pragma unroll
          for (int i = 0; i < 5; ++i) V.b[i * NR + rr] -= db[i];
      }
    } else {
      const int G = NT / nel >= 32 ? 32 : 16;
      const int g = tid / G, gl = tid % G;
      const int lane = tid & 31, gbase = lane & ~(G - 1);
      const unsigned gmask = G == 32 ? 0xffffffffu : (0xffffu << gbase);
      const int r = s * (2 * g + 1);
      if (g < nel) elim_row_grp<NR>(V, Rt, r, s, rhs, G, gl, gbase, gmask, status);
      __syncthreads();
      if (g < nel)
        for (int e = gl; e < 20; e += G) {
          if (e < 15) V.D[e * NR + r + s] -= Rt[e * NR + r];
          else if (rhs) V.b[(e - 15) * NR + r + s] -= Rt[e * NR + r];
        }
    }
    __syncthreads();
  }
}

// forward elimination of a new rhs in b through the stored factors
template <int NR, int NT>
__device__ __forceinline__ void tile_rhs(const TileV &V, int T) {
  const int tid = threadIdx.x;
#pragma unroll 1
  for (int s = 1; s < T; s <<= 1) {
    const int nel = T / (2 * s);
    float db[5];
    int r = -1;
    if (tid < nel) {
      r = s * (2 * tid + 1);
      const int lft = r - s;
      float L[15], v[5], y[5];
#pragma unroll
      for (int i = 0; i < 15; ++i) L[i] = V.D[i * NR + r];
#pragma unroll
      for (int i = 0; i < 5; ++i) v[i] = V.b[i * NR + r];
      fwd5(L, v, y);
#pragma unroll
      for (int i = 0; i < 5; ++i) V.b[i * NR + r] = y[i];
#pragma unroll
      for (int p = 0; p < 5; ++p) {
        float tl = 0.f, tr = 0.f;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
          tl += V.Ya[(5 * i + p) * NR + r] * y[i];
          tr += V.Bm[(5 * i + p) * NR + r] * y[i];
        }
        V.b[p * NR + lft] -= tl;
        db[p] = tr;
      }
    }
    __syncthreads();
    if (r >= 0)
#pragma unroll
      for (int i = 0; i < 5; ++i) V.b[i * NR + r + s] -= db[i];
    __syncthreads();
  }
}

// back-substitution: b holds the multipliers of rows 0 and T and y of the
// eliminated rows; afterwards the multipliers of every row
template <int NR, int NT>
__device__ __forceinline__ void tile_back(const TileV &V, int T) {
  const int tid = threadIdx.x;
#pragma unroll 1
  for (int s = T / 2; s >= 1; s >>= 1) {
    const int nel = T / (2 * s);
    if (tid < nel) {
      const int r = s * (2 * tid + 1);
      float L[15], v[5], x[5], ll[5], lr[5];
#pragma unroll
      for (int i = 0; i < 15; ++i) L[i] = V.D[i * NR + r];
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        ll[i] = V.b[i * NR + r - s];
        lr[i] = V.b[i * NR + r + s];
      }
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        float t = V.b[i * NR + r];
#pragma unroll
        for (int c = 0; c < 5; ++c) t -= V.Ya[(5 * i + c) * NR + r] * ll[c] + V.Bm[(5 * i + c) * NR + r] * lr[c];
        v[i] = t;
      }
      bwd5(L, v, x);
#pragma unroll
      for (int i = 0; i < 5; ++i) V.b[i * NR + r] = x[i];
    }
    __syncthreads();
  }
}

// asynchronous copies global -> shared (sm_80+): 16 bytes (both addresses
// 16-byte aligned) or 4 bytes; completed by cp_async_wait_all
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// ---------------------------------------------------------------------------
// level-0 tiles: per-body and per-joint work of the chain
// ---------------------------------------------------------------------------
struct SegSmem {
  float D[15][SEG_NR];
  float Bm[25][SEG_NR];
  float Ya[25][SEG_NR];
  float b[5][SEG_NR];
  float Rh[9][SEG_NB], Rl[9][SEG_NB];  // R of the tile bodies (double-float)
  float U[12][SEG_NB];                 // u (FIRST), dq0 (CORR)
  float Z[12][SEG_NB];                 // z (CORR)
  float Hh[9][SEG_NR], Hl[9][SEG_NR];  // joint frames R_H of the tile rows (double-float)
};

__device__ __forceinline__ TileV seg_view(SegSmem &sm) {
  return TileV{&sm.D[0][0], &sm.Bm[0][0], &sm.Ya[0][0], &sm.b[0][0]};
}

__device__ __forceinline__ void ld_R_ff(const SegSmem &sm, int i, ff R[9]) {
#pragma unroll
  for (int c = 0; c < 9; ++c) R[c] = ff{sm.Rh[c][i], sm.Rl[c][i]};
}

__device__ __forceinline__ void ld_H_ff(const SegSmem &sm, int i, ff H[9]) {
#pragma unroll
  for (int c = 0; c < 9; ++c) H[c] = ff{sm.Hh[c][i], sm.Hl[c][i]};
}

// Sec. 4.3 in double-float: a = R_a ua, normalised (one Newton step of
// 1/sqrt, the iterate being unit to round-off), its sign chosen so that
// a_y >= 0 (the axis is sign-free), R_H = I + [v]x + [v]x^2 / (1 + a_y),
// v = a x e_y = (-a_z, 0, a_x)
__device__ __forceinline__ void hinge_frame_ff(const ff R[9], const double ua[3], ff H[9]) {
  const ff u0 = ff_from(ua[0]), u1 = ff_from(ua[1]), u2 = ff_from(ua[2]);
  ff a[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) a[r] = ff_fma(R[3 * r], u0, ff_fma(R[3 * r + 1], u1, ff_mul(R[3 * r + 2], u2)));
  const ff n2 = ff_fma(a[0], a[0], ff_fma(a[1], a[1], ff_mul(a[2], a[2])));
  ff sc = ff_sub(ff_make(1.5f), ff_mulf(n2, 0.5f));
  if (a[1].h < 0.f || (a[1].h == 0.f && a[1].l < 0.f)) sc = ff_neg(sc);
#pragma unroll
  for (int r = 0; r < 3; ++r) a[r] = ff_mul(a[r], sc);
  const ff vx = ff_neg(a[2]), vz = a[0];
  const ff k = ff_rcp(ff_add(ff_make(1.f), a[1]));
  const ff kxz = ff_mul(k, ff_mul(vx, vz));
  H[0] = ff_sub(ff_make(1.f), ff_mul(k, ff_mul(vz, vz)));
  H[1] = ff_neg(vz);
  H[2] = kxz;
  H[3] = vz;
  H[4] = ff_sub(ff_make(1.f), ff_mul(k, ff_fma(vx, vx, ff_mul(vz, vz))));
  H[5] = ff_neg(vx);
  H[6] = kxz;
  H[7] = vx;
  H[8] = ff_sub(ff_make(1.f), ff_mul(k, ff_mul(vx, vx)));
}

// A p in double-float for the affine coordinates q (Eq. abd, A(r,c) = q[3c+r])
__device__ __forceinline__ void Ap_ff(const double q[12], const ff p[3], ff out[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
    out[a] = ff_fma(ff_from(q[a]), p[0], ff_fma(ff_from(q[3 + a]), p[1], ff_mul(ff_from(q[6 + a]), p[2])));
}

// gap x_a(pa) - x_b(pb) of a point pair (Eq. ball) as (A_a pa - A_b pb) +
// (t_a - t_b), the translation difference taken in FP64 (exact for
// neighbours) so that a long chain far from the origin keeps the gap at the
// round-off of the body size; without bbody, pb is a world point
__device__ __forceinline__ void gap_ff(const double qa[12], const double pa[3], bool bbody, const double qb[12],
                                       const double pb[3], ff d[3]) {
  const ff pfa[3] = {ff_from(pa[0]), ff_from(pa[1]), ff_from(pa[2])};
  ff la[3];
  Ap_ff(qa, pfa, la);
  if (bbody) {
    const ff pfb[3] = {ff_from(pb[0]), ff_from(pb[1]), ff_from(pb[2])};
    ff lb[3];
    Ap_ff(qb, pfb, lb);
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = ff_add(ff_sub(la[a], lb[a]), ff_from(qa[9 + a] - qb[9 + a]));
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = ff_add(la[a], ff_from(qa[9 + a] - pb[a]));
  }
}

// world displacement R (J(p) x) of rest point p under the rest-frame
// increment x (FP32 values), in double-float
__device__ __forceinline__ void disp_ff(const ff R[9], const float x[12], const ff p[3], ff out[3]) {
  ff l[3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    l[a] = ff_add(ff_fma(ff_make(x[a]), p[0], ff_fma(ff_make(x[3 + a]), p[1], ff_mul(ff_make(x[6 + a]), p[2]))),
                  ff_make(x[9 + a]));
#pragma unroll
  for (int a = 0; a < 3; ++a) out[a] = ff_fma(R[3 * a], l[0], ff_fma(R[3 * a + 1], l[1], ff_mul(R[3 * a + 2], l[2])));
}

// rows of a joint from world vectors at its points: ball rows 0-2 = g1;
// hinge rows 0-2 = R_H g1, rows 3, 4 = the x and z rows of R_H times g2
__device__ __forceinline__ void rows_ff(bool hinge, const ff H[9], const ff g1[3], const ff g2[3], ff out[5]) {
  if (!hinge) {
    out[0] = g1[0];
    out[1] = g1[1];
    out[2] = g1[2];
    out[3] = ff_make(0.f);
    out[4] = ff_make(0.f);
    return;
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) out[r] = ff_fma(H[3 * r], g1[0], ff_fma(H[3 * r + 1], g1[1], ff_mul(H[3 * r + 2], g1[2])));
  out[3] = ff_fma(H[0], g2[0], ff_fma(H[1], g2[1], ff_mul(H[2], g2[2])));
  out[4] = ff_fma(H[6], g2[0], ff_fma(H[7], g2[1], ff_mul(H[8], g2[2])));
}

// the same in FP32 for one body side (s = +1 on body a, -1 on b): the rows
// of G_side x for the rest-frame vector x of that body
__device__ __forceinline__ void side_rows_f(bool hinge, float s, const float R[9], const float H[9], const float x[12],
                                            const float p1[3], const float p2[3], float out[5]) {
  float w[3];
  disp_at(R, x, p1, w);
  if (!hinge) {
    out[0] = s * w[0];
    out[1] = s * w[1];
    out[2] = s * w[2];
    out[3] = 0.f;
    out[4] = 0.f;
    return;
  }
#pragma unroll
  for (int r = 0; r < 3; ++r) out[r] = s * (H[3 * r] * w[0] + H[3 * r + 1] * w[1] + H[3 * r + 2] * w[2]);
  disp_at(R, x, p2, w);
  out[3] = s * (H[0] * w[0] + H[1] * w[1] + H[2] * w[2]);
  out[4] = s * (H[6] * w[0] + H[7] * w[1] + H[8] * w[2]);
}

// joint points of one side in FP32 (p2 only for hinges)
__device__ __forceinline__ void side_points_f(const DevJoints &J, int k, bool side_a, bool hinge, float p1[3],
                                              float p2[3]) {
  load3f(side_a ? J.pa1f : J.pb1f, J.K, k, p1);
  if (hinge) load3f(side_a ? J.pa2f : J.pb2f, J.K, k, p2);
  else p2[0] = p2[1] = p2[2] = 0.f;
}

__device__ __forceinline__ void side_points_ff(const DevJoints &J, int k, bool side_a, bool hinge, ff p1[3],
                                               ff p2[3]) {
  double d[3];
  load3(side_a ? J.pa1 : J.pb1, J.K, k, d);
#pragma unroll
  for (int a = 0; a < 3; ++a) p1[a] = ff_from(d[a]);
  if (hinge) {
    load3(side_a ? J.pa2 : J.pb2, J.K, k, d);
#pragma unroll
    for (int a = 0; a < 3; ++a) p2[a] = ff_from(d[a]);
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a) p2[a] = ff_make(0.f);
  }
}

// rest-frame directions of a joint's rows on one body (columns of E):
// ball: s R^T; hinge: s R^T R_H^T (the rows of R_H)
__device__ __forceinline__ void side_dirs(bool hinge, float s, const float R[9], const float H[9], float E[3][3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int r = 0; r < 3; ++r)
      E[a][r] = hinge ? s * (R[a] * H[3 * r] + R[3 + a] * H[3 * r + 1] + R[6 + a] * H[3 * r + 2]) : s * R[3 * r + a];
}

// a joint's diagonal block from one body: E^T Mbar(p, p') E per point pair
// (Eq. chain-Schur-blocks through the body's 3x3 point compliances)
__device__ __forceinline__ void self_block(const float h[16], bool hinge, const float E[3][3], const float p1[3],
                                           const float p2[3], float Dp[15]) {
  const int c012[3] = {0, 1, 2}, c02[3] = {0, 2, 0};
  float Mb[3][3], blk[3][3];
#pragma unroll
  for (int i = 0; i < 15; ++i) Dp[i] = 0.f;
  mbar(h, p1, p1, Mb);
  project<3, 3>(E, c012, Mb, E, c012, blk);
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c <= r; ++c) Dp[pk5(r, c)] = blk[r][c];
  if (hinge) {
    mbar(h, p2, p1, Mb);
    project<2, 3>(E, c02, Mb, E, c012, blk);
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) Dp[pk5(3 + r, c)] = blk[r][c];
    mbar(h, p2, p2, Mb);
    project<2, 2>(E, c02, Mb, E, c02, blk);
    Dp[pk5(3, 3)] = blk[0][0];
    Dp[pk5(4, 3)] = blk[1][0];
    Dp[pk5(4, 4)] = blk[1][1];
  }
}

// coupling of the body's lower joint (rows) with its upper joint (columns)
__device__ __forceinline__ void couple_block(const float h[16], bool h0, const float E0[3][3], const float p01[3],
                                             const float p02[3], bool h1, const float E1[3][3], const float p11[3],
                                             const float p12[3], float Bp[25]) {
  const int c012[3] = {0, 1, 2}, c02[3] = {0, 2, 0};
  float Mb[3][3], blk[3][3];
#pragma unroll
  for (int i = 0; i < 25; ++i) Bp[i] = 0.f;
  mbar(h, p01, p11, Mb);
  project<3, 3>(E0, c012, Mb, E1, c012, blk);
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) Bp[5 * r + c] = blk[r][c];
  if (h1) {
    mbar(h, p01, p12, Mb);
    project<3, 2>(E0, c012, Mb, E1, c02, blk);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 2; ++c) Bp[5 * r + 3 + c] = blk[r][c];
  }
  if (h0) {
    mbar(h, p02, p11, Mb);
    project<2, 3>(E0, c02, Mb, E1, c012, blk);
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) Bp[5 * (3 + r) + c] = blk[r][c];
    if (h1) {
      mbar(h, p02, p12, Mb);
      project<2, 2>(E0, c02, Mb, E1, c02, blk);
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) Bp[5 * (3 + r) + 3 + c] = blk[r][c];
    }
  }
}

// One thread per chain body (path order): R = polar(A) (Eq. polar), the
// rest-frame rhs fbar (Sec. 3.3, Eq. module1-wrench-map) and u = Hbar^{-1}
// fbar (Eq. abd_final, FP32), and fbar - Hbar u, the residual of that FP32
// solve, from double-float arithmetic; for each joint whose body a this is,
// the hinge frame R_H (Sec. 4.3, from body a) and C(q_n) (Eq. ball / hinge),
// the gap taken against the other body's (or the world's) points.
__global__ void __launch_bounds__(128, 4) k_seg_body(DevBodies B, DevJoints J, StepParams p, SegChain S,
                                                     int *status) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= S.nb) return;
  const int M = B.M, K = J.K;
  double qa[12], qv[12], cst[6];
#pragma unroll
  for (int i = 0; i < 12; ++i) qa[i] = B.q[(size_t)i * M + j];
#pragma unroll
  for (int i = 0; i < 12; ++i) qv[i] = B.qd[(size_t)i * M + j];
  cst[0] = ldg(B.sig + j);
  cst[1] = ldg(B.sig + M + j);
  cst[2] = ldg(B.sig + 2 * (size_t)M + j);
  cst[3] = ldg(B.mass + j);
  cst[4] = ldg(B.vmu + j);
  cst[5] = ldg(B.vlam + j);
  ff A[9], R[9];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int r = 0; r < 3; ++r) A[3 * r + c] = ff_from(qa[3 * c + r]);
  int nit = 0;
  const int st = polar3_ff(A, R, &nit);
  if (S.polar_iters) count_add(S.polar_iters, (unsigned)nit);
  if (st) {
    set_status(status, st);
#pragma unroll
    for (int i = 0; i < 9; ++i) R[i] = ff_make((i % 4 == 0) ? 1.0f : 0.0f);
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    B.Rf[(size_t)i * M + j] = R[i].h;
    B.Rlo[(size_t)i * M + j] = R[i].l;
  }
  {
    ff qd[12], fb[12], uf[12], hu[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) qd[i] = ff_from(qv[i]);
    fbar_ff(A, R, qd, cst, p, fb);
    float hf[16], v[12], u[12];
    load_hinvf(B, j, hf);
#pragma unroll
    for (int i = 0; i < 12; ++i) v[i] = fb[i].h;
    hinv_apply_t(hf, v, u);
#pragma unroll
    for (int i = 0; i < 12; ++i) uf[i] = ff_make(u[i]);
    const ff s3[3] = {ff_from(cst[0]), ff_from(cst[1]), ff_from(cst[2])};
    const ff ih = ff_from(p.inv_h);
    hbar_apply_ff(s3, ff_from(cst[3]), ff_from(cst[4]), ff_from(cst[5]), ff_mul(ih, ih), uf, hu);
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      S.u[(size_t)i * S.nb + j] = u[i];
      S.rf[(size_t)i * S.nb + j] = ff_sub(fb[i], hu[i]).h;
    }
  }
  // the joints of which this body is body a: its lower joint j - sigma (this
  // body being the joint's upper body) and its upper joint j + 1 - sigma
#pragma unroll 1
  for (int sd = 0; sd < 2; ++sd) {
    const int k = j + sd - S.sigma;
    if (k < 0 || k >= K) continue;
    const uint8_t f = __ldg(S.cjf + k);
    const bool mine = sd == 0 ? ((f & SEGJ_UP) && !(f & SEGJ_A_LO)) : ((f & SEGJ_LO) && (f & SEGJ_A_LO));
    if (!mine) continue;
    const bool hinge = (f & SEGJ_HINGE) != 0;
    ff H[9];
    if (hinge) {
      double ua[3];
      load3(J.ua, K, k, ua);
      hinge_frame_ff(R, ua, H);
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        J.RHf[(size_t)i * K + k] = H[i].h;
        S.RHlo[(size_t)i * K + k] = H[i].l;
      }
      if (S.write_cj)
#pragma unroll
        for (int i = 0; i < 9; ++i) J.RH[(size_t)i * K + k] = ff_to(H[i]);
    }
    // the other body: the lower path body of the lower joint, the upper one
    // of the upper joint (absent: a world point)
    const bool bbody = (f & (sd == 0 ? SEGJ_LO : SEGJ_UP)) != 0;
    const int ob = sd == 0 ? j - 1 : j + 1;
    double qb[12], pa[3], pb[3];
    load12(B.q, M, bbody ? ob : j, qb);
    ff g1[3], g2[3], c[5];
    load3(J.pa1, K, k, pa);
    load3(J.pb1, K, k, pb);
    gap_ff(qa, pa, bbody, qb, pb, g1);
    if (hinge) {
      load3(J.pa2, K, k, pa);
      load3(J.pb2, K, k, pb);
      gap_ff(qa, pa, bbody, qb, pb, g2);
    }
    rows_ff(hinge, H, g1, g2, c);
#pragma unroll
    for (int r = 0; r < 5; ++r) J.c[(size_t)r * K + k] = (r < 3 || hinge) ? ff_to(c[r]) : 0.0;
  }
}

// body and row of the tile phases: thread t takes its own item, and threads
// 0 and 1 a second one (tile bodies 0 and SEG_T + 1; tile row SEG_T, the
// next tile's first row, goes to thread 0)
__device__ __forceinline__ int seg_body_of(int tid, int round) {
  return round == 0 ? tid + 1 : (tid == 0 ? 0 : (tid == 1 ? SEG_T + 1 : -1));
}
__device__ __forceinline__ int seg_row_of(int tid, int round) { return round == 0 ? tid : (tid == 0 ? SEG_T : -1); }

// One CTA per tile of SEG_T joints; the pass is MODE (see the file comment).
template <int MODE>
__global__ void __launch_bounds__(SEG_NT, SEG_MINB) k_seg(DevBodies B, DevJoints J, StepParams p, SegChain S,
                                                    int *status) {
  extern __shared__ __align__(16) unsigned char seg_raw[];
  SegSmem &sm = *reinterpret_cast<SegSmem *>(seg_raw);
  const TileV V = seg_view(sm);
  const int tid = threadIdx.x;
  const int t = blockIdx.x;
  const int P0 = S.lv0.N;
  const int k0 = t * SEG_T;
  const int K = J.K, M = B.M, nb = S.nb;
  const int gb0 = k0 - 1 + S.sigma;  // path index of tile body 0
  const double rr = p.residual_rhs ? 1.0 : 0.0;

  // ---- later passes: the tile's factors (FIRST stored them) and the
  // forward-eliminated rhs of its eliminated rows, copied asynchronously
  // while the tile's bodies and rows are read
  if (MODE != SEG_FIRST) {
    const float *src = S.fac + (size_t)t * SEG_FAC;
    float *dst = &sm.D[0][0];
    for (int i = tid; i < SEG_FAC / 4; i += SEG_NT) cp_async16(dst + 4 * i, src + 4 * i);
    if (tid >= 1) {
      if (k0 + tid < K) {
#pragma unroll
        for (int r = 0; r < 5; ++r) cp_async4(&sm.b[r][tid], S.ytile + (size_t)r * K + k0 + tid);
      } else {
#pragma unroll
        for (int r = 0; r < 5; ++r) sm.b[r][tid] = 0.f;
      }
    }
    if (MODE == SEG_FINAL) {
      // the own body's dq0 and z, the rows' approximate multipliers
      const int gbi = gb0 + tid + 1;
      if (gbi < nb)
#pragma unroll
        for (int i = 0; i < 12; ++i) {
          cp_async4(&sm.U[i][tid + 1], S.dq0 + (size_t)i * nb + gbi);
          cp_async4(&sm.Z[i][tid + 1], S.z + (size_t)i * nb + gbi);
        }
      if (k0 + tid < K)
#pragma unroll
        for (int r = 0; r < 5; ++r) cp_async4(&sm.Rl[r][tid], S.lam0 + (size_t)r * K + k0 + tid);
    }
    cp_async_commit();
  }

  // ---- tile bodies: rotation; tile rows: block storage and frames
#pragma unroll 1
  for (int round = 0; round < 2; ++round) {
    const int bi = seg_body_of(tid, round);
    const int gbi = gb0 + bi;
    if (bi >= 0 && gbi >= 0 && gbi < nb) {
#pragma unroll
      for (int i = 0; i < 9; ++i) sm.Rh[i][bi] = B.Rf[(size_t)i * M + gbi];
      if (MODE == SEG_CORR)
#pragma unroll
        for (int i = 0; i < 9; ++i) sm.Rl[i][bi] = B.Rlo[(size_t)i * M + gbi];
    }
    const int ji = seg_row_of(tid, round);
    if (ji >= 0) {
      const int kj = k0 + ji;
      const bool jex = kj < K;
      const bool jh = jex && (__ldg(S.cjf + kj) & SEGJ_HINGE);
      if (MODE == SEG_FIRST) {
#pragma unroll
        for (int i = 0; i < 15; ++i) sm.D[i][ji] = 0.f;
        if (ji < SEG_T) {
          // padded rows of a ball, and rows past the last joint, carry an identity diagonal
          if (!jh) {
            sm.D[pk5(3, 3)][ji] = 1.f;
            sm.D[pk5(4, 4)][ji] = 1.f;
          }
          if (!jex) {
            sm.D[pk5(0, 0)][ji] = 1.f;
            sm.D[pk5(1, 1)][ji] = 1.f;
            sm.D[pk5(2, 2)][ji] = 1.f;
          }
        }
#pragma unroll
        for (int i = 0; i < 25; ++i) sm.Bm[i][ji] = 0.f;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
          sm.b[i][ji] = 0.f;
          (&sm.Z[0][0])[i * SEG_NR + ji] = 0.f;  // the rows' sums of G u (FIRST) start at zero
        }
      }
      if (MODE == SEG_CORR)
#pragma unroll
        for (int i = 0; i < 15; ++i) (&sm.U[0][0])[i * SEG_NR + ji] = 0.f;
      if (jh) {
#pragma unroll
        for (int i = 0; i < 9; ++i) sm.Hh[i][ji] = J.RHf[(size_t)i * K + kj];
        if (MODE == SEG_CORR)
#pragma unroll
          for (int i = 0; i < 9; ++i) sm.Hl[i][ji] = S.RHlo[(size_t)i * K + kj];
      }
    }
  }
  __syncthreads();

  // ---- FIRST: b = G u + C(q_n) (FP32 products).  Each body forms the rows
  // of G u on its two joints (its sides), added into the rows' sums Es in
  // two barrier phases (upper joint, then lower joint); body SEG_T's side of
  // the next tile's first row is that row's FP64 part dl, and row 0's lower
  // side (body 0) the previous tile's (tile 0 owns its body 0).  Then each
  // row adds C(q_n): row 0 in FP64 (b0), the others into b.
  if (MODE == SEG_FIRST) {
    float *Es = &sm.Z[0][0];  // [5][SEG_NR]
    float elo[2][5];
    int erow[2] = {-1, -1};
#pragma unroll
    for (int round = 0; round < 2; ++round) {
      const int bi = round == 0 ? tid + 1 : ((tid == 0 && t == 0) ? 0 : -1);
      const int gbi = gb0 + bi;
      if (bi < 0 || gbi < 0 || gbi >= nb) continue;
      float Rf[9], u[12];
#pragma unroll
      for (int i = 0; i < 9; ++i) Rf[i] = sm.Rh[i][bi];
#pragma unroll
      for (int i = 0; i < 12; ++i) u[i] = S.u[(size_t)i * nb + gbi];
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        // sd 0: the upper joint (row bi, this body its lower body); sd 1: the lower joint (row bi - 1)
        const int row = bi - sd;
        const int k = k0 + row;
        float e[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        bool has = row >= 0 && k < K;
        uint8_t f = 0;
        if (has) {
          f = __ldg(S.cjf + k);
          has = (f & (sd == 0 ? SEGJ_LO : SEGJ_UP)) != 0;
        }
        if (has) {
          const bool hg = (f & SEGJ_HINGE) != 0;
          const bool side_a = sd == 0 ? (f & SEGJ_A_LO) != 0 : !(f & SEGJ_A_LO);
          float Hf[9], p1[3], p2[3];
#pragma unroll
          for (int i = 0; i < 9; ++i) Hf[i] = hg ? sm.Hh[i][row] : 0.f;
          side_points_f(J, k, side_a, hg, p1, p2);
          side_rows_f(hg, side_a ? 1.f : -1.f, Rf, Hf, u, p1, p2, e);
        }
        if (sd == 0) {
          if (row == SEG_T) {
#pragma unroll
            for (int r = 0; r < 5; ++r) S.lv0.r[0].dl[(size_t)r * P0 + t] = f2d(e[r]);
          } else if (has) {
#pragma unroll
            for (int r = 0; r < 5; ++r) Es[r * SEG_NR + row] += e[r];
          }
        } else if (has) {
#pragma unroll
          for (int r = 0; r < 5; ++r) elo[round][r] = e[r];
          erow[round] = row;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int round = 0; round < 2; ++round)
      if (erow[round] >= 0)
#pragma unroll
        for (int r = 0; r < 5; ++r) Es[r * SEG_NR + erow[round]] += elo[round][r];
    __syncthreads();
    const int kj = k0 + tid;
    if (kj < K) {
      const bool jh = (__ldg(S.cjf + kj) & SEGJ_HINGE) != 0;
      const int nr = jh ? 5 : 3;
      double c[5];
#pragma unroll
      for (int r = 0; r < 5; ++r) c[r] = r < nr ? rr * J.c[(size_t)r * K + kj] : 0.0;
      if (tid == 0) {
#pragma unroll
        for (int r = 0; r < 5; ++r) S.lv0.r[0].b0[(size_t)r * P0 + t] = c[r] + f2d(Es[r * SEG_NR]);
      } else {
#pragma unroll
        for (int r = 0; r < 5; ++r) sm.b[r][tid] = r < nr ? d2f(c[r]) + Es[r * SEG_NR + tid] : 0.f;
      }
    }
  }

  // ---- FIRST: Gram blocks and the tile's factorization; the later passes
  // read the factors FIRST stored
  if (MODE == SEG_FIRST) {
    // ---- Gram blocks of the tile bodies 0 .. SEG_T: for body i, its lower
    // joint i - 1 and upper joint i (as tile rows); D += per-body parts, the
    // coupling of the two joints into the lower joint's row
    float Dlow[2][15];
    int lrow[2] = {-1, -1};
#pragma unroll
    for (int round = 0; round < 2; ++round) {
      const int bi = round == 0 ? tid + 1 : (tid == 0 ? 0 : -1);
      const int gbi = gb0 + bi;
      if (bi < 0 || gbi < 0 || gbi >= nb) continue;
      const int jl = bi - 1, ju = bi;
      const int kl = k0 + jl, ku = k0 + ju;
      const bool has_l = jl >= 0 && kl < K && (__ldg(S.cjf + kl) & SEGJ_UP);
      const bool has_u = ku < K && (__ldg(S.cjf + ku) & SEGJ_LO);
      if (!has_l && !has_u) continue;
      float Rf[9], h[16];
#pragma unroll
      for (int i = 0; i < 9; ++i) Rf[i] = sm.Rh[i][bi];
      load_hinvf(B, gbi, h);
      float E0[3][3], E1[3][3], p01[3], p02[3], p11[3], p12[3];
      bool h0 = false, h1 = false;
      if (has_l) {
        const uint8_t f = __ldg(S.cjf + kl);
        h0 = (f & SEGJ_HINGE) != 0;
        const bool side_a = !(f & SEGJ_A_LO);  // this body is the joint's upper body
        float Hf[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) Hf[i] = h0 ? sm.Hh[i][jl] : 0.f;
        side_points_f(J, kl, side_a, h0, p01, p02);
        side_dirs(h0, side_a ? 1.f : -1.f, Rf, Hf, E0);
        self_block(h, h0, E0, p01, p02, Dlow[round]);
        lrow[round] = jl;
      }
      if (has_u) {
        const uint8_t f = __ldg(S.cjf + ku);
        h1 = (f & SEGJ_HINGE) != 0;
        const bool side_a = (f & SEGJ_A_LO) != 0;  // this body is the joint's lower body
        float Hf[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) Hf[i] = h1 ? sm.Hh[i][ju] : 0.f;
        side_points_f(J, ku, side_a, h1, p11, p12);
        side_dirs(h1, side_a ? 1.f : -1.f, Rf, Hf, E1);
        if (ju < SEG_T) {
          float Dp[15];
          self_block(h, h1, E1, p11, p12, Dp);
#pragma unroll
          for (int i = 0; i < 15; ++i) sm.D[i][ju] += Dp[i];
        }
      }
      if (has_l && has_u) {
        float Bp[25];
        couple_block(h, h0, E0, p01, p02, h1, E1, p11, p12, Bp);
#pragma unroll
        for (int i = 0; i < 25; ++i) sm.Bm[i][jl] = Bp[i];
      }
    }
    __syncthreads();
#pragma unroll
    for (int round = 0; round < 2; ++round)
      if (lrow[round] >= 0)
#pragma unroll
        for (int i = 0; i < 15; ++i) sm.D[i][lrow[round]] += Dlow[round][i];
    __syncthreads();

    tile_factor<SEG_NR, SEG_NT>(V, &sm.U[0][0], SEG_T, true, status);
    // the factors of the tile (D, Bm, Ya: whole 16-byte words) for the later passes
    {
      const float4 *src = reinterpret_cast<const float4 *>(&sm.D[0][0]);
      float4 *dst = reinterpret_cast<float4 *>(S.fac + (size_t)t * SEG_FAC);
      for (int i = tid; i < SEG_FAC / 4; i += SEG_NT) dst[i] = src[i];
    }
  }

  if (MODE == SEG_FIRST) {
    // the tile's first row and what it adds to the next tile's first row
    SegLevel L = S.lv0;
    if (tid < 15) {
      L.Dn[(size_t)tid * P0 + t] = sm.D[tid][0];
      L.Da[(size_t)tid * P0 + t] = sm.D[tid][SEG_T];
    }
    if (tid < 25) L.Bn[(size_t)tid * P0 + t] = sm.Bm[tid][0];
    if (tid < 5) {
      L.r[0].bn[(size_t)tid * P0 + t] = sm.b[tid][0];
      L.r[0].ba[(size_t)tid * P0 + t] = sm.b[tid][SEG_T];
    }
    if (tid >= 1 && k0 + tid < K)
#pragma unroll
      for (int r = 0; r < 5; ++r) S.ytile[(size_t)r * K + k0 + tid] = sm.b[r][tid];
    return;
  }

  // ---- back-substitution: the first rows' multipliers from the level above
  {
    const float *lam_up = S.lv0.r[MODE == SEG_CORR ? 0 : 1].lam;
    if (tid < 5) {
      sm.b[tid][0] = lam_up[(size_t)tid * P0 + t];
      sm.b[tid][SEG_T] = t + 1 < P0 ? lam_up[(size_t)tid * P0 + t + 1] : 0.f;
    }
  }
  cp_async_wait_all();
  __syncthreads();
  tile_back<SEG_NR, SEG_NT>(V, SEG_T);

  if (MODE == SEG_CORR) {
    if (k0 + tid < K)
#pragma unroll
      for (int r = 0; r < 5; ++r) S.lam0[(size_t)r * K + k0 + tid] = sm.b[r][tid];
    // ---- own bodies: dq0 = u - Hbar^{-1} g(lambda0), the primal residual
    // r_p = fbar - Hbar dq0 - g = (fbar - Hbar u) + (Hbar (u - dq0) - g)
    // with the second bracket in double-float, z = Hbar^{-1} r_p
    // the rows' sums of the sides (RD: G dq0 as double-float pairs, GZ: G z),
    // zeroed with the tile rows
    float *RDh = &sm.U[0][0], *RDl = RDh + 5 * SEG_NR, *GZ = RDh + 10 * SEG_NR;
    ff rdl[2][5];
    float gzl[2][5];
    int lrow[2] = {-1, -1};
#pragma unroll
    for (int round = 0; round < 2; ++round) {
      const int bi = round == 0 ? tid + 1 : ((tid == 0 && t == 0) ? 0 : -1);
      const int gbi = gb0 + bi;
      if (bi < 0 || gbi < 0 || gbi >= nb) continue;
      const int jl = bi - 1, ju = bi;
      const int kl = k0 + jl, ku = k0 + ju;
      const uint8_t fl = (jl >= 0 && kl < K) ? __ldg(S.cjf + kl) : (uint8_t)0;
      const uint8_t fu = (ku < K) ? __ldg(S.cjf + ku) : (uint8_t)0;
      const bool hl = jl >= 0 && (fl & SEGJ_UP), hu = (fu & SEGJ_LO) != 0;
      ff R[9];
      ld_R_ff(sm, bi, R);
      ff g[12];
#pragma unroll
      for (int i = 0; i < 12; ++i) g[i] = ff_make(0.f);
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        const bool has = sd == 0 ? hl : hu;
        if (!has) continue;
        const int row = sd == 0 ? jl : ju;
        const int k = sd == 0 ? kl : ku;
        const uint8_t f = sd == 0 ? fl : fu;
        const bool hg = (f & SEGJ_HINGE) != 0;
        const bool side_a = sd == 0 ? !(f & SEGJ_A_LO) : (f & SEGJ_A_LO) != 0;
        ff p1[3], p2[3], H[9], l[5];
        side_points_ff(J, k, side_a, hg, p1, p2);
#pragma unroll
        for (int r = 0; r < 5; ++r) l[r] = ff_make(sm.b[r][row]);
        ff F1[3], F2[3];
        if (hg) {
          ld_H_ff(sm, row, H);
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            F1[a] = ff_fma(H[a], l[0], ff_fma(H[3 + a], l[1], ff_mul(H[6 + a], l[2])));
            F2[a] = ff_fma(H[a], l[3], ff_mul(H[6 + a], l[4]));
          }
        } else {
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            F1[a] = l[a];
            F2[a] = ff_make(0.f);
          }
        }
#pragma unroll
        for (int pt = 0; pt < 2; ++pt) {
          if (pt == 1 && !hg) break;
          ff f3[3], P[3];
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const ff Fa0 = pt == 0 ? F1[0] : F2[0], Fa1 = pt == 0 ? F1[1] : F2[1], Fa2 = pt == 0 ? F1[2] : F2[2];
            f3[a] = ff_fma(R[a], Fa0, ff_fma(R[3 + a], Fa1, ff_mul(R[6 + a], Fa2)));
            if (!side_a) f3[a] = ff_neg(f3[a]);
            P[a] = pt == 0 ? p1[a] : p2[a];
          }
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            g[a] = ff_fma(P[0], f3[a], g[a]);
            g[3 + a] = ff_fma(P[1], f3[a], g[3 + a]);
            g[6 + a] = ff_fma(P[2], f3[a], g[6 + a]);
            g[9 + a] = ff_add(g[9 + a], f3[a]);
          }
        }
      }
      float hf[16], v[12], w[12], dq0[12], z[12];
      load_hinvf(B, gbi, hf);
#pragma unroll
      for (int i = 0; i < 12; ++i) v[i] = g[i].h;
      hinv_apply_t(hf, v, w);
      // dq0 is the FP32 difference u - w as rounded; the residual is taken
      // at that dq0: Hbar dq0 = Hbar u - Hbar (u - dq0), with u - dq0 exact
      // as a double-float pair
      ff wf[12], hw[12];
#pragma unroll
      for (int i = 0; i < 12; ++i) {
        const float ui = S.u[(size_t)i * nb + gbi];
        dq0[i] = ui - w[i];
        wf[i] = ff_sub(ff_make(ui), ff_make(dq0[i]));
      }
      const ff s3[3] = {ff_from(ldg(B.sig + gbi)), ff_from(ldg(B.sig + M + gbi)),
                        ff_from(ldg(B.sig + 2 * (size_t)M + gbi))};
      const ff ih = ff_from(p.inv_h);
      hbar_apply_ff(s3, ff_from(ldg(B.mass + gbi)), ff_from(ldg(B.vmu + gbi)), ff_from(ldg(B.vlam + gbi)),
                    ff_mul(ih, ih), wf, hw);
#pragma unroll
      for (int i = 0; i < 12; ++i) v[i] = S.rf[(size_t)i * nb + gbi] + ff_sub(hw[i], g[i]).h;
      hinv_apply_t(hf, v, z);
#pragma unroll
      for (int i = 0; i < 12; ++i) {
        S.dq0[(size_t)i * nb + gbi] = dq0[i];
        S.z[(size_t)i * nb + gbi] = z[i];
      }
      // this body's sides of its two joints: rows of G dq0 (double-float)
      // and of G z (FP32); sd 0: the upper joint (row bi, this body its lower
      // body), added at once; sd 1: the lower joint (row bi - 1), after the
      // barrier; body SEG_T's upper side is the next tile's first row's
      float Rf[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) Rf[i] = R[i].h;
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        const int row = bi - sd;
        const int k = k0 + row;
        bool has = row >= 0 && k < K;
        uint8_t f = 0;
        if (has) {
          f = __ldg(S.cjf + k);
          has = (f & (sd == 0 ? SEGJ_LO : SEGJ_UP)) != 0;
        }
        const bool hg = (f & SEGJ_HINGE) != 0;
        ff rd[5];
        float gz[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int r = 0; r < 5; ++r) rd[r] = ff_make(0.f);
        if (has) {
          const bool side_a = sd == 0 ? (f & SEGJ_A_LO) != 0 : !(f & SEGJ_A_LO);
          ff H[9], p1[3], p2[3], x1[3], x2[3];
          float Hf[9], pf1[3], pf2[3];
          if (hg) {
            ld_H_ff(sm, row, H);
#pragma unroll
            for (int i = 0; i < 9; ++i) Hf[i] = H[i].h;
          } else {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
              H[i] = ff_make(0.f);
              Hf[i] = 0.f;
            }
          }
          side_points_ff(J, k, side_a, hg, p1, p2);
          disp_ff(R, dq0, p1, x1);
          if (hg) disp_ff(R, dq0, p2, x2);
          else x2[0] = x2[1] = x2[2] = ff_make(0.f);
          if (!side_a)
#pragma unroll
            for (int a3 = 0; a3 < 3; ++a3) {
              x1[a3] = ff_neg(x1[a3]);
              x2[a3] = ff_neg(x2[a3]);
            }
          rows_ff(hg, H, x1, x2, rd);
          side_points_f(J, k, side_a, hg, pf1, pf2);
          side_rows_f(hg, side_a ? 1.f : -1.f, Rf, Hf, z, pf1, pf2, gz);
        }
        if (sd == 0 && row == SEG_T) {
          const int nr = hg ? 5 : 3;
#pragma unroll
          for (int r = 0; r < 5; ++r) {
            S.lv0.r[1].dl[(size_t)r * P0 + t] = r < nr ? ff_to(rd[r]) : 0.0;
            sm.b[r][SEG_T] = gz[r];
          }
        } else if (sd == 0 && has) {
#pragma unroll
          for (int r = 0; r < 5; ++r) {
            const ff o = ff_add(ff{RDh[r * SEG_NR + row], RDl[r * SEG_NR + row]}, rd[r]);
            RDh[r * SEG_NR + row] = o.h;
            RDl[r * SEG_NR + row] = o.l;
            GZ[r * SEG_NR + row] += gz[r];
          }
        } else if (sd == 1 && has) {
#pragma unroll
          for (int r = 0; r < 5; ++r) {
            rdl[round][r] = rd[r];
            gzl[round][r] = gz[r];
          }
          lrow[round] = row;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int round = 0; round < 2; ++round)
      if (lrow[round] >= 0) {
        const int row = lrow[round];
#pragma unroll
        for (int r = 0; r < 5; ++r) {
          const ff o = ff_add(ff{RDh[r * SEG_NR + row], RDl[r * SEG_NR + row]}, rdl[round][r]);
          RDh[r * SEG_NR + row] = o.h;
          RDl[r * SEG_NR + row] = o.l;
          GZ[r * SEG_NR + row] += gzl[round][r];
        }
      }
    __syncthreads();
    // ---- rows: r_d = C(q_n) + G dq0 (double-float), rhs G z + r_d; row 0's
    // own part in FP64 (b0), its G z part into b
    double worst = 0.0;
    {
      const int kj = k0 + tid;
      if (kj < K) {
        const bool jh = (__ldg(S.cjf + kj) & SEGJ_HINGE) != 0;
        const int nr = jh ? 5 : 3;
        ff rd[5];
#pragma unroll
        for (int r = 0; r < 5; ++r)
          rd[r] = r < nr ? ff_add(ff{RDh[r * SEG_NR + tid], RDl[r * SEG_NR + tid]},
                                  ff_from(rr * J.c[(size_t)r * K + kj]))
                         : ff_make(0.f);
        if (tid == 0) {
#pragma unroll
          for (int r = 0; r < 5; ++r) {
            S.lv0.r[1].b0[(size_t)r * P0 + t] = r < nr ? ff_to(rd[r]) : 0.0;
            sm.b[r][0] = r < nr ? GZ[r * SEG_NR] : 0.f;
          }
        } else {
#pragma unroll
          for (int r = 0; r < 5; ++r) {
            sm.b[r][tid] = r < nr ? rd[r].h + GZ[r * SEG_NR + tid] : 0.f;
            if (r < nr) worst = fmax(worst, fabs(ff_to(rd[r])));
          }
        }
      } else {
#pragma unroll
        for (int r = 0; r < 5; ++r) sm.b[r][tid] = 0.f;
      }
    }
    if (S.refine_max) {
      for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
      if ((tid & 31) == 0) atomic_max_nonneg(S.refine_max, worst);
    }
    __syncthreads();
    tile_rhs<SEG_NR, SEG_NT>(V, SEG_T);
    SegLevel L = S.lv0;
    if (tid < 5) {
      L.r[1].bn[(size_t)tid * P0 + t] = sm.b[tid][0];
      L.r[1].ba[(size_t)tid * P0 + t] = sm.b[tid][SEG_T];
    }
    if (tid >= 1 && k0 + tid < K)
#pragma unroll
      for (int r = 0; r < 5; ++r) S.ytile[(size_t)r * K + k0 + tid] = sm.b[r][tid];
    return;
  }

  // ---- FINAL: multipliers, then the state update of the tile's own bodies
  if (k0 + tid < K) {
    const int kj = k0 + tid;
#pragma unroll
    for (int r = 0; r < 5; ++r)
      J.lambda[(size_t)r * K + kj] = f2d(sm.Rl[r][tid]) + f2d(sm.b[r][tid]);
  }
#pragma unroll 1
  for (int round = 0; round < 2; ++round) {
    const int bi = round == 0 ? tid + 1 : ((tid == 0 && t == 0) ? 0 : -1);
    const int gbi = gb0 + bi;
    if (bi < 0 || gbi < 0 || gbi >= nb) continue;
    const int jl = bi - 1, ju = bi;
    const int kl = k0 + jl, ku = k0 + ju;
    const uint8_t fl = (jl >= 0 && kl < K) ? __ldg(S.cjf + kl) : (uint8_t)0;
    const uint8_t fu = (ku < K) ? __ldg(S.cjf + ku) : (uint8_t)0;
    const bool hl = jl >= 0 && (fl & SEGJ_UP), hu = (fu & SEGJ_LO) != 0;
    float Rf[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) Rf[i] = sm.Rh[i][bi];
    // g = diag4(R^T) sum_k G_kj^T dlambda_k (FP32)
    float g[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) g[i] = 0.f;
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      const bool has = sd == 0 ? hl : hu;
      if (!has) continue;
      const int row = sd == 0 ? jl : ju;
      const int k = sd == 0 ? kl : ku;
      const uint8_t f = sd == 0 ? fl : fu;
      const bool hg = (f & SEGJ_HINGE) != 0;
      const bool side_a = sd == 0 ? !(f & SEGJ_A_LO) : (f & SEGJ_A_LO) != 0;
      const float sg = side_a ? 1.f : -1.f;
      float p1[3], p2[3], l[5], F1[3], F2[3];
      side_points_f(J, k, side_a, hg, p1, p2);
#pragma unroll
      for (int r = 0; r < 5; ++r) l[r] = sm.b[r][row];
      if (hg) {
        float H[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) H[i] = sm.Hh[i][row];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          F1[a] = H[a] * l[0] + H[3 + a] * l[1] + H[6 + a] * l[2];
          F2[a] = H[a] * l[3] + H[6 + a] * l[4];
        }
      } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          F1[a] = l[a];
          F2[a] = 0.f;
        }
      }
#pragma unroll
      for (int pt = 0; pt < 2; ++pt) {
        if (pt == 1 && !hg) break;
        float f3[3], P[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const float F0 = pt == 0 ? F1[0] : F2[0], Fb = pt == 0 ? F1[1] : F2[1], Fc = pt == 0 ? F1[2] : F2[2];
          f3[a] = sg * (Rf[a] * F0 + Rf[3 + a] * Fb + Rf[6 + a] * Fc);
          P[a] = pt == 0 ? p1[a] : p2[a];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          g[a] += P[0] * f3[a];
          g[3 + a] += P[1] * f3[a];
          g[6 + a] += P[2] * f3[a];
          g[9 + a] += f3[a];
        }
      }
    }
    float hf[16], w[12];
    load_hinvf(B, gbi, hf);
    hinv_apply_t(hf, g, w);
    ff dq[12], R[9];
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      const float d0 = bi > 0 ? sm.U[i][bi] : S.dq0[(size_t)i * nb + gbi];
      const float zi = bi > 0 ? sm.Z[i][bi] : S.z[(size_t)i * nb + gbi];
      dq[i] = ff_add(ff_make(d0), ff_make(zi - w[i]));
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) R[i] = ff{Rf[i], B.Rlo[(size_t)i * M + gbi]};
    const ff ih = ff_from(p.inv_h);
#pragma unroll
    for (int blk = 0; blk < 4; ++blk)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const ff d = ff_fma(R[3 * a], dq[3 * blk], ff_fma(R[3 * a + 1], dq[3 * blk + 1], ff_mul(R[3 * a + 2], dq[3 * blk + 2])));
        const size_t o = (size_t)(3 * blk + a) * M + gbi;
        B.q[o] += ff_to(d);
        B.qd[o] = ff_to(ff_mul(d, ih));
      }
  }
}

// ---------------------------------------------------------------------------
// upper systems: row r of the system of a level's tile outputs
// ---------------------------------------------------------------------------
__device__ __forceinline__ void up_row(const SegLevel &L, const SegRhs &R, int r, float D[15], float Bm[25],
                                       float b[5], double &worst) {
  const int N = L.N;
  if (r >= N) {
#pragma unroll
    for (int i = 0; i < 15; ++i) D[i] = 0.f;
#pragma unroll
    for (int i = 0; i < 5; ++i) D[pk5(i, i)] = 1.f;
#pragma unroll
    for (int i = 0; i < 25; ++i) Bm[i] = 0.f;
#pragma unroll
    for (int i = 0; i < 5; ++i) b[i] = 0.f;
    return;
  }
#pragma unroll
  for (int i = 0; i < 15; ++i) D[i] = L.Dn[(size_t)i * N + r] + (r > 0 ? L.Da[(size_t)i * N + r - 1] : 0.f);
#pragma unroll
  for (int i = 0; i < 25; ++i) Bm[i] = r + 1 < N ? L.Bn[(size_t)i * N + r] : 0.f;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    float v = R.bn[(size_t)i * N + r] + (r > 0 ? R.ba[(size_t)i * N + r - 1] : 0.f);
    if (R.b0) {
      const double e = R.b0[(size_t)i * N + r] + (r > 0 ? R.dl[(size_t)i * N + r - 1] : 0.0);
      worst = fmax(worst, fabs(e));
      v += d2f(e);
    }
    b[i] = v;
  }
}

struct UpSmem {
  float D[15][UP_NR];
  float Bm[25][UP_NR];
  float Ya[25][UP_NR];
  float b[5][UP_NR];
  float Rt[20][UP_NR];  // right-neighbour updates of the group eliminations
};

// rows r0 .. r0 + T - 1 of `in` into the tile (identity past the last row),
// row T the accumulator of the external row
__device__ __forceinline__ double up_load(UpSmem &sm, const SegLevel &in, const SegRhs &rin, int r0, int T) {
  double worst = 0.0;
  for (int i = threadIdx.x; i <= T; i += UP_NT) {
    float D[15], Bm[25], b[5];
    if (i < T) {
      up_row(in, rin, r0 + i, D, Bm, b, worst);
    } else {
#pragma unroll
      for (int c = 0; c < 15; ++c) D[c] = 0.f;
#pragma unroll
      for (int c = 0; c < 25; ++c) Bm[c] = 0.f;
#pragma unroll
      for (int c = 0; c < 5; ++c) b[c] = 0.f;
    }
#pragma unroll
    for (int c = 0; c < 15; ++c) sm.D[c][i] = D[c];
#pragma unroll
    for (int c = 0; c < 25; ++c) sm.Bm[c][i] = Bm[c];
#pragma unroll
    for (int c = 0; c < 5; ++c) sm.b[c][i] = b[c];
  }
  __syncthreads();
  return worst;
}

__device__ __forceinline__ void worst_out(double worst, unsigned long long *rmax) {
  if (!rmax) return;
  for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(rmax, worst);
}

__global__ void __launch_bounds__(UP_NT) k_seg_up_reduce(SegLevel in, SegRhs rin, SegLevel out, SegRhs rout,
                                                         int T, int write_db, unsigned long long *rmax,
                                                         int *status) {
  extern __shared__ __align__(16) unsigned char up_raw[];
  UpSmem &sm = *reinterpret_cast<UpSmem *>(up_raw);
  const TileV V{&sm.D[0][0], &sm.Bm[0][0], &sm.Ya[0][0], &sm.b[0][0]};
  const int t = blockIdx.x, P = out.N;
  worst_out(up_load(sm, in, rin, t * T, T), rmax);
  tile_factor<UP_NR, UP_NT>(V, &sm.Rt[0][0], T, true, status);
  const int tid = threadIdx.x;
  if (write_db) {
    if (tid < 15) {
      out.Dn[(size_t)tid * P + t] = sm.D[tid][0];
      out.Da[(size_t)tid * P + t] = sm.D[tid][T];
    }
    if (tid < 25) out.Bn[(size_t)tid * P + t] = sm.Bm[tid][0];
  }
  if (tid < 5) {
    rout.bn[(size_t)tid * P + t] = sm.b[tid][0];
    rout.ba[(size_t)tid * P + t] = sm.b[tid][T];
  }
}

// the whole system (in.N <= T rows) in one CTA
__global__ void __launch_bounds__(UP_NT) k_seg_up_top(SegLevel in, SegRhs rin, int T, unsigned long long *rmax,
                                                      int *status) {
  extern __shared__ __align__(16) unsigned char up_raw[];
  UpSmem &sm = *reinterpret_cast<UpSmem *>(up_raw);
  const TileV V{&sm.D[0][0], &sm.Bm[0][0], &sm.Ya[0][0], &sm.b[0][0]};
  worst_out(up_load(sm, in, rin, 0, T), rmax);
  tile_factor<UP_NR, UP_NT>(V, &sm.Rt[0][0], T, true, status);
  const int tid = threadIdx.x;
  if (tid == 0) {
    float L[15], v[5], y[5], x[5];
#pragma unroll
    for (int i = 0; i < 15; ++i) L[i] = sm.D[i][0];
    chol5(L, status);
#pragma unroll
    for (int i = 0; i < 5; ++i) v[i] = sm.b[i][0];
    fwd5(L, v, y);
    bwd5(L, y, x);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      sm.b[i][0] = x[i];
      sm.b[i][T] = 0.f;
    }
  }
  __syncthreads();
  tile_back<UP_NR, UP_NT>(V, T);
  const int N = in.N;
  for (int i = tid; i < N; i += UP_NT)
#pragma unroll
    for (int c = 0; c < 5; ++c) rin.lam[(size_t)c * N + i] = sm.b[c][i];
}

// the rows of tile t of `in` given the multipliers of the tiles' first rows
// (next's solution): the tile's factorization and forward elimination again,
// then back-substitution
__global__ void __launch_bounds__(UP_NT) k_seg_up_back(SegLevel in, SegRhs rin, int T, int P,
                                                       const float *lam_next, int *status) {
  extern __shared__ __align__(16) unsigned char up_raw[];
  UpSmem &sm = *reinterpret_cast<UpSmem *>(up_raw);
  const TileV V{&sm.D[0][0], &sm.Bm[0][0], &sm.Ya[0][0], &sm.b[0][0]};
  const int t = blockIdx.x, N = in.N;
  up_load(sm, in, rin, t * T, T);
  tile_factor<UP_NR, UP_NT>(V, &sm.Rt[0][0], T, true, status);
  const int tid = threadIdx.x;
  if (tid < 5) {
    sm.b[tid][0] = lam_next[(size_t)tid * P + t];
    sm.b[tid][T] = t + 1 < P ? lam_next[(size_t)tid * P + t + 1] : 0.f;
  }
  __syncthreads();
  tile_back<UP_NR, UP_NT>(V, T);
  for (int i = tid; i < T; i += UP_NT) {
    const int r = t * T + i;
    if (r < N)
#pragma unroll
      for (int c = 0; c < 5; ++c) rin.lam[(size_t)c * N + r] = sm.b[c][i];
  }
}

// ---------------------------------------------------------------------------
cudaError_t seg_init() {
  cudaError_t e;
  e = cudaFuncSetAttribute(k_seg<SEG_FIRST>, cudaFuncAttributeMaxDynamicSharedMemorySize, sizeof(SegSmem));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_seg<SEG_CORR>, cudaFuncAttributeMaxDynamicSharedMemorySize, sizeof(SegSmem));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_seg<SEG_FINAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, sizeof(SegSmem));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_seg_up_reduce, cudaFuncAttributeMaxDynamicSharedMemorySize, sizeof(UpSmem));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_seg_up_top, cudaFuncAttributeMaxDynamicSharedMemorySize, sizeof(UpSmem));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_seg_up_back, cudaFuncAttributeMaxDynamicSharedMemorySize, sizeof(UpSmem));
}

void launch_seg_body(const DevBodies &B, const DevJoints &J, const StepParams &p, const SegChain &S, int *status,
                     cudaStream_t s) {
  if (S.nb > 0) k_seg_body<<<(S.nb + 127) / 128, 128, 0, s>>>(B, J, p, S, status);
}

void launch_seg_tiles(int mode, const DevBodies &B, const DevJoints &J, const StepParams &p, const SegChain &S,
                      int *status, cudaStream_t s) {
  const int P0 = S.lv0.N;
  if (P0 <= 0) return;
  const size_t sh = sizeof(SegSmem);
  if (mode == SEG_FIRST) k_seg<SEG_FIRST><<<P0, SEG_NT, sh, s>>>(B, J, p, S, status);
  else if (mode == SEG_CORR) k_seg<SEG_CORR><<<P0, SEG_NT, sh, s>>>(B, J, p, S, status);
  else k_seg<SEG_FINAL><<<P0, SEG_NT, sh, s>>>(B, J, p, S, status);
}

void launch_seg_up_reduce(const SegLevel &in, const SegLevel &out, int T, int pass, bool write_db,
                          unsigned long long *rmax, int *status, cudaStream_t s) {
  k_seg_up_reduce<<<out.N, UP_NT, sizeof(UpSmem), s>>>(in, in.r[pass], out, out.r[pass], T, write_db ? 1 : 0,
                                                        rmax, status);
}

void launch_seg_up_top(const SegLevel &in, int T, int pass, unsigned long long *rmax, int *status,
                       cudaStream_t s) {
  k_seg_up_top<<<1, UP_NT, sizeof(UpSmem), s>>>(in, in.r[pass], T, rmax, status);
}

void launch_seg_up_back(const SegLevel &in, const SegLevel &next, int T, int pass, int *status, cudaStream_t s) {
  k_seg_up_back<<<next.N, UP_NT, sizeof(UpSmem), s>>>(in, in.r[pass], T, next.N, next.r[pass].lam, status);
}

}  // namespace mabd
