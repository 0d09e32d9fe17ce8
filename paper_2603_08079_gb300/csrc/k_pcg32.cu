// FP32 preconditioned conjugate gradients on the dual S x = rhs with
// S = G H^{-1} G^T (Eq. dual), matrix-free as in the FP64 graph path, for
// the mixed-precision form: every product in FP32 from the FP32 copies of R,
// Hbar^{-1}, the joint points and the hinge frames; dot products are summed
// per thread in FP32 and across threads and blocks in FP64, in a fixed
// order.  The FP64 residual-correction sweeps of the mixed form call one
// such solve per sweep (from x = 0), so each solve only has to reduce its
// own residual by the inner tolerance.
//
// Two drivers run the same per-body and per-joint steps: one launch per
// step of an iteration (host-paced), and a persistent cooperative kernel
// that keeps the whole solve on the device, the phases separated by a grid
// barrier whose waits are bounded (k_p32_persist).
#include "grid_sync.cuh"
#include "lpc_apply.cuh"
#include "mabd_f32.cuh"

namespace mabd {

__device__ __forceinline__ int pkf(int r, int c) { return r >= c ? r * (r + 1) / 2 + c : c * (c + 1) / 2 + r; }

// z = D^{-1} r with the packed Cholesky factor (reciprocal diagonal)
__device__ __forceinline__ void dsolve(const float L[15], int C, const float r[5], float z[5]) {
  float y[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    float t = i < C ? r[i] : 0.f;
#pragma unroll
    for (int q = 0; q < i; ++q) t -= L[pkf(i, q)] * y[q];
    y[i] = t * L[pkf(i, i)];
  }
#pragma unroll
  for (int i = 4; i >= 0; --i) {
    float t = y[i];
#pragma unroll
    for (int q = i + 1; q < 5; ++q) t -= L[pkf(q, i)] * z[q];
    z[i] = i < C ? t * L[pkf(i, i)] : 0.f;
  }
}

// t_k = C_k r_k (rows 0-2) with C packed lower (c00 c10 c11 c20 c21 c22)
__device__ __forceinline__ void ctimes(const float *Cp, const float r[5], float *t, int K, int k) {
  t[k] = Cp[0] * r[0];
  t[(size_t)K + k] = Cp[1] * r[0] + Cp[2] * r[1];
  t[2 * (size_t)K + k] = Cp[3] * r[0] + Cp[4] * r[1] + Cp[5] * r[2];
}

// ---------------------------------------------------------------------------
// per-joint and per-body steps
// ---------------------------------------------------------------------------
// setup of joint k: D_k in FP32 and its Cholesky factor; x = 0, r = rhs,
// p = 0 and z = D^{-1} r (block Jacobi) or t = C r (learned); adds r.z (block
// Jacobi) and r.r to the thread's sums
template <bool XJ>
__device__ __forceinline__ void p32_setup_one(const DevBodies &B, const DevJoints &J, const DevPCG32 &P,
                                              const double *rhs, int *status, int k, float &rz, float &rr) {
  const int K = J.K;
  const int C = joint_nrows(J.type[k]);
  const uint8_t fl = J.flags[k];
  float D[15];
#pragma unroll
  for (int i = 0; i < 15; ++i) D[i] = 0.f;
  for (int side = 0; side < 2; ++side) {
    if (!(fl & (side == 0 ? JF_A_FREE : JF_B_FREE))) continue;
    const int j = side == 0 ? J.ja[k] : J.jb[k];
    float R[9], h[16], E[5][3], PR[5][3], WR[5];
    load_Rf(B, j, R);
    load_hf(B, j, h);
    rows_pt_f<XJ>(J, k, side, R, E, PR, WR);
    float W[5][12], Z[5][12];
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      if (r >= C) break;
      const float *pp = PR[r];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        W[r][a] = pp[0] * E[r][a];
        W[r][3 + a] = pp[1] * E[r][a];
        W[r][6 + a] = pp[2] * E[r][a];
        W[r][9 + a] = WR[r] * E[r][a];
      }
      hinvf_apply(h, W[r], Z[r]);
    }
#pragma unroll
    for (int r = 0; r < 5; ++r)
#pragma unroll
      for (int t = 0; t <= r; ++t) {
        if (r >= C) continue;
        float v = 0.f;
#pragma unroll
        for (int a = 0; a < 12; ++a) v += W[r][a] * Z[t][a];
        D[pkf(r, t)] += v;
      }
  }
  // Cholesky with reciprocal diagonal
  bool ok = true;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    float sum = c < C ? D[pkf(c, c)] : 1.f;
#pragma unroll
    for (int q = 0; q < c; ++q) sum -= D[pkf(c, q)] * D[pkf(c, q)];
    if (!(sum > 0.f)) {
      if (c < C) ok = false;
      sum = 1.f;
    }
    const float id = rsqrtf(sum);
    D[pkf(c, c)] = id;
#pragma unroll
    for (int r = c + 1; r < 5; ++r) {
      float t = r < C ? D[pkf(r, c)] : 0.f;
#pragma unroll
      for (int q = 0; q < c; ++q) t -= D[pkf(r, q)] * D[pkf(c, q)];
      D[pkf(r, c)] = t * id;
    }
  }
  if (!ok) set_status(status, ST_NOT_SPD);
#pragma unroll
  for (int i = 0; i < 15; ++i) P.Lpre[(size_t)i * K + k] = D[i];
  float rv[5], z[5];
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    rv[r] = r < C ? (float)rhs[(size_t)r * K + k] : 0.f;
    const size_t o = (size_t)r * K + k;
    P.r[o] = rv[r];
    P.p[o] = 0.f;
    P.x[o] = 0.f;
  }
  if (P.t) {
    ctimes(P.Cl + (size_t)6 * k, rv, P.t, K, k);
#pragma unroll
    for (int r = 0; r < 5; ++r) rr += rv[r] * rv[r];
  } else {
    dsolve(D, C, rv, z);
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      P.z[(size_t)r * K + k] = z[r];
      rz += rv[r] * z[r];
      rr += rv[r] * rv[r];
    }
  }
}

// body j: zb_j = Hbar^{-1} sum_rows p_r W_r with p = z + beta p_old
template <bool XJ>
__device__ __forceinline__ void p32_body_one(const DevBodies &B, const DevJoints &J, const DevIncidence &I,
                                             const DevPCG32 &P, int j, float beta) {
  const int K = J.K, M = B.M;
  float R[9], g[12];
  load_Rf(B, j, R);
#pragma unroll
  for (int a = 0; a < 12; ++a) g[a] = 0.f;
  for (int e = I.off[j]; e < I.off[j + 1]; ++e) {
    const int k = I.joint[e];
    float E[5][3], PR[5][3], WR[5];
    const int C = rows_pt_f<XJ>(J, k, I.side[e], R, E, PR, WR);
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      if (r >= C) break;
      const float pr = P.z[(size_t)r * K + k] + beta * P.p[(size_t)r * K + k];
      const float *pp = PR[r];
      const float w = WR[r];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float v = pr * E[r][a];
        g[a] += pp[0] * v;
        g[3 + a] += pp[1] * v;
        g[6 + a] += pp[2] * v;
        g[9 + a] += w * v;
      }
    }
  }
  float h[16], z[12];
  load_hf(B, j, h);
  hinvf_apply(h, g, z);
#pragma unroll
  for (int a = 0; a < 12; ++a) P.zb[(size_t)a * M + j] = z[a];
}

// joint k: p = z + beta p_old (stored), Sp = sum_bodies W zb; returns p.Sp
template <bool XJ>
__device__ __forceinline__ float p32_joint_sp_one(const DevBodies &B, const DevJoints &J, const DevPCG32 &P,
                                                  int k, float beta) {
  const int K = J.K;
  const int C = joint_nrows(J.type[k]);
  const uint8_t fl = J.flags[k];
  float pv[5], sp[5];
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    pv[r] = r < C ? P.z[(size_t)r * K + k] + beta * P.p[(size_t)r * K + k] : 0.f;
    sp[r] = 0.f;
  }
  for (int side = 0; side < 2; ++side) {
    if (!(fl & (side == 0 ? JF_A_FREE : JF_B_FREE))) continue;
    const int j = side == 0 ? J.ja[k] : J.jb[k];
    float R[9], E[5][3], PR[5][3], zb[12], WR[5];
    load_Rf(B, j, R);
    rows_pt_f<XJ>(J, k, side, R, E, PR, WR);
#pragma unroll
    for (int a = 0; a < 12; ++a) zb[a] = P.zb[(size_t)a * B.M + j];
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      if (r >= C) break;
      const float *pp = PR[r];
      const float w = WR[r];
      float v = 0.f;
#pragma unroll
      for (int a = 0; a < 3; ++a)
        v += E[r][a] * (pp[0] * zb[a] + pp[1] * zb[3 + a] + pp[2] * zb[6 + a] + w * zb[9 + a]);
      sp[r] += v;
    }
  }
  float psp = 0.f;
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    P.p[(size_t)r * K + k] = pv[r];
    P.Sp[(size_t)r * K + k] = sp[r];
    psp += pv[r] * sp[r];
  }
  return psp;
}

// joint k: x += alpha p, r -= alpha Sp, then z = D^{-1} r (block Jacobi) or
// t = C r (learned); adds r.z (block Jacobi) and r.r to the thread's sums
__device__ __forceinline__ void p32_update_one(const DevJoints &J, const DevPCG32 &P, int k, float alpha,
                                               float &rz, float &rr) {
  const int K = J.K;
  const int C = joint_nrows(J.type[k]);
  float rv[5], L[15], z[5];
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const size_t o = (size_t)r * K + k;
    P.x[o] += alpha * P.p[o];
    rv[r] = P.r[o] - alpha * P.Sp[o];
    P.r[o] = rv[r];
  }
  if (P.t) {
    ctimes(P.Cl + (size_t)6 * k, rv, P.t, K, k);
#pragma unroll
    for (int r = 0; r < 5; ++r) rr += rv[r] * rv[r];
  } else {
#pragma unroll
    for (int i = 0; i < 15; ++i) L[i] = P.Lpre[(size_t)i * K + k];
    dsolve(L, C, rv, z);
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      P.z[(size_t)r * K + k] = z[r];
      rz += rv[r] * z[r];
      rr += rv[r] * rv[r];
    }
  }
}

// ---------------------------------------------------------------------------
// one launch per step of an iteration
// ---------------------------------------------------------------------------
// block-level sums of two per-thread values into part[blockIdx], part[nb + blockIdx]
__device__ __forceinline__ void block_partials(double a, double b, double *part, int nb) {
  __shared__ double s1[128], s2[128];
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s1[0];
    part[nb + blockIdx.x] = s2[0];
  }
}

__device__ __forceinline__ void block_sum2_32(const double *part, int n, int nb, double &a, double &b) {
  __shared__ double s1[P32_THREADS], s2[P32_THREADS];
  double x = 0.0, y = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    x += part[i];
    y += part[nb + i];
  }
  s1[threadIdx.x] = x;
  s2[threadIdx.x] = y;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
    }
    __syncthreads();
  }
  a = s1[0];
  b = s2[0];
}

template <bool XJ>
__global__ void __launch_bounds__(128) k_p32_setup(DevBodies B, DevJoints J, DevPCG32 P,
                                                   const double *rhs, int *status) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  float rz = 0.f, rr = 0.f;
  if (k < J.K) p32_setup_one<XJ>(B, J, P, rhs, status, k, rz, rr);
  block_partials((double)rz, (double)rr, P.part, P.nblocks);
}

__global__ void k_p32_setup_reduce(DevPCG32 P, double rtol) {
  double rz, rr;
  block_sum2_32(P.part, P.nblocks, P.nblocks, rz, rr);
  if (threadIdx.x == 0) {
    P.scal[0] = rz;
    P.scal[2] = 0.0;
    P.scal[3] = rr;
    P.scal[4] = rr;
    P.scal[5] = rtol * rtol;
    P.iter[0] = 0;
    P.iter[1] = (rr == 0.0) ? 1 : 0;
  }
}

template <bool XJ>
__global__ void __launch_bounds__(128) k_p32_body(DevBodies B, DevJoints J, DevIncidence I, DevPCG32 P) {
  if (P.iter[1]) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= B.M || B.fixed[j]) return;
  p32_body_one<XJ>(B, J, I, P, j, (float)P.scal[2]);
}

template <bool XJ>
__global__ void __launch_bounds__(128) k_p32_joint_sp(DevBodies B, DevJoints J, DevPCG32 P) {
  if (P.iter[1]) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const float psp = k < J.K ? p32_joint_sp_one<XJ>(B, J, P, k, (float)P.scal[2]) : 0.f;
  block_partials((double)psp, 0.0, P.part, P.nblocks);
}

__global__ void k_p32_alpha(DevPCG32 P) {
  if (P.iter[1]) return;
  double psp, dummy;
  block_sum2_32(P.part, P.nblocks, P.nblocks, psp, dummy);
  if (threadIdx.x == 0) {
    P.scal[6] = psp;
    P.scal[1] = psp > 0.0 ? P.scal[0] / psp : 0.0;
  }
}

__global__ void __launch_bounds__(128) k_p32_joint_update(DevJoints J, DevPCG32 P) {
  if (P.iter[1]) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  float rz = 0.f, rr = 0.f;
  if (k < J.K) p32_update_one(J, P, k, (float)P.scal[1], rz, rr);
  block_partials((double)rz, (double)rr, P.part, P.nblocks);
}

__global__ void k_p32_beta(DevPCG32 P, int max_iters) {
  if (P.iter[1]) return;
  double rz, rr;
  block_sum2_32(P.part, P.nblocks, P.nblocks, rz, rr);
  if (threadIdx.x == 0) {
    const double rz_old = P.scal[0];
    P.scal[2] = rz_old != 0.0 ? rz / rz_old : 0.0;
    P.scal[0] = rz;
    P.scal[3] = rr;
    const int it = P.iter[0] + 1;
    P.iter[0] = it;
    if (rr <= P.scal[5] * P.scal[4] || it >= max_iters) P.iter[1] = 1;
  }
}

__global__ void __launch_bounds__(128) k_p32_finish(DevJoints J, DevPCG32 P, double *out, double *acc) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int K = J.K;
  if (k >= K) return;
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const size_t o = (size_t)r * K + k;
    const double v = (double)P.x[o];
    out[o] = v;
    if (acc) acc[o] += v;
  }
}

// ---------------------------------------------------------------------------
// persistent solve: one cooperative launch per solve
// ---------------------------------------------------------------------------
// The iterations of an FP32 PCG solve in one launch, from the state that
// the setup kernels left (grid-stride loops over joints and bodies; partial
// sums per block in P.ppart: [0] r.z, [1] r.r, [2] p.Sp).  LPC: the learned
// preconditioner (P.t set), whose application takes two more barriers.
// Writes out = x (FP64), acc += x when given, and P.scal / P.iter as the
// one-launch-per-step driver does.
template <bool XJ, bool LPC>
__global__ void __launch_bounds__(P32_THREADS, 3)
    k_p32_persist(DevBodies B, DevJoints J, DevIncidence I, DevPCG32 P, LpcGraph G, LpcAct A, int max_iters,
                  double *out, double *acc, int *status) {
  __shared__ double sh[P32_THREADS];
  const unsigned nblk = gridDim.x;
  const int tid = blockIdx.x * P32_THREADS + threadIdx.x, nth = nblk * P32_THREADS;
  const int K = J.K, M = B.M;
  double *prz = P.ppart, *prr = P.ppart + P32_MAXB, *ppsp = P.ppart + 2 * P32_MAXB;
  unsigned gen = 0;
  bool ok = true;
  // from the state k_p32_setup and k_p32_setup_reduce left
  double rz = P.scal[0], rr = P.scal[3];
  const double bb = P.scal[4], tol2 = P.scal[5];
  double beta = 0.0;
  int it = 0;
  bool done = P.iter[1] != 0;
  while (ok && !done && it < max_iters) {
    for (int j = tid; j < M; j += nth)
      if (!B.fixed[j]) p32_body_one<XJ>(B, J, I, P, j, (float)beta);
    ok = grid_barrier(P.bar, nblk, gen);
    if (!ok) break;
    float psp = 0.f;
    for (int k = tid; k < K; k += nth) psp += p32_joint_sp_one<XJ>(B, J, P, k, (float)beta);
    const double bpsp = block_sum((double)psp, sh);
    if (threadIdx.x == 0) ppsp[blockIdx.x] = bpsp;
    ok = grid_barrier(P.bar, nblk, gen);
    if (!ok) break;
    const double pSp = grid_sum(ppsp, nblk, sh);
    const double alpha = pSp > 0.0 ? rz / pSp : 0.0;
    float rzf = 0.f, rrf = 0.f;
    for (int k = tid; k < K; k += nth) p32_update_one(J, P, k, (float)alpha, rzf, rrf);
    const double brr = block_sum((double)rrf, sh);
    if (LPC) {
      if (threadIdx.x == 0) prr[blockIdx.x] = brr;
      ok = grid_barrier(P.bar, nblk, gen);
      if (!ok) break;
      for (int k = tid; k < K; k += nth) lpc_y_one(G, A, P.t, P.y, k);
      ok = grid_barrier(P.bar, nblk, gen);
      if (!ok) break;
      for (int k = tid; k < K; k += nth) rzf += lpc_z_one(G, A, P.y, P.r, P.z, k);
      const double brz = block_sum((double)rzf, sh);
      if (threadIdx.x == 0) prz[blockIdx.x] = brz;
    } else {
      const double brz = block_sum((double)rzf, sh);
      if (threadIdx.x == 0) {
        prz[blockIdx.x] = brz;
        prr[blockIdx.x] = brr;
      }
    }
    ok = grid_barrier(P.bar, nblk, gen);
    if (!ok) break;
    const double rz_new = grid_sum(prz, nblk, sh);
    rr = grid_sum(prr, nblk, sh);
    beta = rz != 0.0 ? rz_new / rz : 0.0;
    rz = rz_new;
    ++it;
    done = rr <= tol2 * bb;
  }
  if (!ok) {
    if (tid == 0) set_status(status, ST_TIMEOUT);
    return;
  }
  for (int k = tid; k < K; k += nth)
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      const size_t o = (size_t)r * K + k;
      const double v = (double)P.x[o];
      out[o] = v;
      if (acc) acc[o] += v;
    }
  __syncthreads();  // every thread of block 0 has read P.scal / P.iter
  if (tid == 0) {
    P.scal[0] = rz;
    P.scal[3] = rr;
    P.iter[0] = it;
    P.iter[1] = 1;
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
void launch_p32_setup(const DevBodies &B, const DevJoints &J, const DevPCG32 &P, const double *rhs,
                      double rtol, int *status, cudaStream_t s, const LpcGraph *lg, const LpcAct *la) {
  if (J.xj) k_p32_setup<true><<<P.nblocks, 128, 0, s>>>(B, J, P, rhs, status);
  else k_p32_setup<false><<<P.nblocks, 128, 0, s>>>(B, J, P, rhs, status);
  if (P.t) launch_lpc_apply(*lg, *la, P.t, P.y, P.r, P.z, P.part, P.nblocks, s, nullptr);
  k_p32_setup_reduce<<<1, P32_THREADS, 0, s>>>(P, rtol);
}

void launch_p32_iteration(const DevBodies &B, const DevJoints &J, const DevIncidence &I,
                          const DevPCG32 &P, int max_iters, cudaStream_t s, const LpcGraph *lg,
                          const LpcAct *la) {
  if (J.xj) {
    k_p32_body<true><<<(B.M + 127) / 128, 128, 0, s>>>(B, J, I, P);
    k_p32_joint_sp<true><<<P.nblocks, 128, 0, s>>>(B, J, P);
  } else {
    k_p32_body<false><<<(B.M + 127) / 128, 128, 0, s>>>(B, J, I, P);
    k_p32_joint_sp<false><<<P.nblocks, 128, 0, s>>>(B, J, P);
  }
  k_p32_alpha<<<1, P32_THREADS, 0, s>>>(P);
  k_p32_joint_update<<<P.nblocks, 128, 0, s>>>(J, P);
  if (P.t) launch_lpc_apply(*lg, *la, P.t, P.y, P.r, P.z, P.part, P.nblocks, s, P.iter);
  k_p32_beta<<<1, P32_THREADS, 0, s>>>(P, max_iters);
}

void launch_p32_finish(const DevJoints &J, const DevPCG32 &P, double *out, double *acc, cudaStream_t s) {
  if (J.K > 0) k_p32_finish<<<(J.K + 127) / 128, 128, 0, s>>>(J, P, out, acc);
}

template <bool XJ, bool LPC>
static void *persist_fn() {
  return (void *)k_p32_persist<XJ, LPC>;
}

int p32_persist_blocks(bool xj, bool lpc) {
  void *f = xj ? (lpc ? persist_fn<true, true>() : persist_fn<true, false>())
               : (lpc ? persist_fn<false, true>() : persist_fn<false, false>());
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, f, P32_THREADS, 0) != cudaSuccess) return 0;
  return std::min(sms * per, P32_MAXB);
}

cudaError_t launch_p32_persist(const DevBodies &B, const DevJoints &J, const DevIncidence &I, const DevPCG32 &P,
                               const LpcGraph *lg, const LpcAct *la, const double *rhs, double rtol,
                               int max_iters, double *out, double *acc, int *status, int nblocks, cudaStream_t s) {
  const bool lpc = P.t != nullptr;
  LpcGraph G{};
  LpcAct A{};
  if (lpc) {
    G = *lg;
    A = *la;
  }
  launch_p32_setup(B, J, P, rhs, rtol, status, s, lg, la);
  cudaError_t e = cudaMemsetAsync(P.bar, 0, 4 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  void *args[] = {(void *)&B, (void *)&J, (void *)&I, (void *)&P, (void *)&G, (void *)&A,
                  (void *)&max_iters, (void *)&out, (void *)&acc, (void *)&status};
  void *f = J.xj ? (lpc ? persist_fn<true, true>() : persist_fn<true, false>())
                 : (lpc ? persist_fn<false, true>() : persist_fn<false, false>());
  return cudaLaunchCooperativeKernel(f, dim3(nblocks), dim3(P32_THREADS), args, 0, s);
}

}  // namespace mabd
