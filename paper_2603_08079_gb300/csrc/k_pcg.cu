// Graph path of one M-ABD step (FP64): the dual system S lambda = b with
// S = G H^{-1} G^T (Eq. dual) solved by conjugate gradients preconditioned
// with the diagonal blocks D_k of S (block Jacobi), matrix-free: S p is
// formed per body as H_j^{-1} G_j^T p (Eq. abd_final) and gathered per joint.
// The closed-loop / irregular case of Sec. 5.5 (the paper relaxes it by
// multi-directional block Gauss-Seidel; CG reaches the exact dual solution).
//
// One iteration = five launches; every kernel returns at once when the
// device flag says the iteration has converged or reached its cap, so the
// host can enqueue several iterations between checks without any waiting.
#include "mabd_device.cuh"

namespace mabd {

constexpr int PCG_THREADS = 256;

__device__ __forceinline__ int pk5(int r, int c) { return r >= c ? r * (r + 1) / 2 + c : c * (c + 1) / 2 + r; }

// rows of joint k on one of its free bodies, with that body's Hbar^{-1}
// applied: W[r] = [p;1] (x) s R^T d_r and Z[r] = Hbar^{-1} W[r]
template <bool XJ>
__device__ __forceinline__ int joint_side_rows(const DevBodies &B, const DevJoints &J, int k, int side,
                                               double W[5][12]) {
  const int j = side == 0 ? J.ja[k] : J.jb[k];
  double R[9], E[5][3], PR[5][3], WR[5];
  load_R(B.R, B.M, j, R);
  const int C = joint_rows_pt<double, XJ>(J, k, side, R, E, PR, WR);
#pragma unroll
  for (int r = 0; r < 5; ++r)
    if (r < C) kron_row_w(PR[r], WR[r], E[r], W[r]);
  const int type = J.type[k];
  if (J.qf && side == 0 && (type == 1 || (XJ && type == 3))) {
    // MABD_JACOBIAN_FULL: the frame term of each row on body a
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      double qh[3];
      load_qf(J.qf, J.K, k, r, qh);
      add_skew_force(qh, 1.0, W[r]);
    }
  }
  return C;
}

// per joint: D_k = sum_j G_kj H_j^{-1} G_kj^T, its Cholesky factor, and the
// start of the iteration: lambda = 0, r = b, z = D^{-1} r, p = 0, rz = r.z
template <bool XJ>
__global__ void __launch_bounds__(128) k_pcg_setup(DevBodies B, DevJoints J, DevPCG P, int *status) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int K = J.K;
  double rz = 0.0, rr = 0.0;
  if (k < K) {
    const int C = joint_nrows(J.type[k]);
    const uint8_t fl = J.flags[k];
    double D[15];
#pragma unroll
    for (int i = 0; i < 15; ++i) D[i] = 0.0;
    for (int side = 0; side < 2; ++side) {
      if (!(fl & (side == 0 ? JF_A_FREE : JF_B_FREE))) continue;
      const int j = side == 0 ? J.ja[k] : J.jb[k];
      double W[5][12], h[16];
      joint_side_rows<XJ>(B, J, k, side, W);
      load_hinv(B, j, h);
      for (int t = 0; t < C; ++t) {
        double z[12];
        hinv_apply(h, W[t], z);
        for (int r = t; r < C; ++r) {
          double v = 0.0;
#pragma unroll
          for (int a = 0; a < 12; ++a) v += W[r][a] * z[a];
          D[pk5(r, t)] += v;
        }
      }
    }
    // Cholesky in place
    for (int c = 0; c < C; ++c) {
      double s = D[pk5(c, c)];
      for (int q = 0; q < c; ++q) s -= D[pk5(c, q)] * D[pk5(c, q)];
      if (!(s > 0.0)) {
        set_status(status, ST_NOT_SPD);
        s = 1.0;
      }
      const double d = sqrt(s);
      D[pk5(c, c)] = d;
      for (int r = c + 1; r < C; ++r) {
        double t = D[pk5(r, c)];
        for (int q = 0; q < c; ++q) t -= D[pk5(r, q)] * D[pk5(c, q)];
        D[pk5(r, c)] = t / d;
      }
    }
#pragma unroll
    for (int i = 0; i < 15; ++i) P.Lpre[(size_t)i * K + k] = D[i];
    double rv[5], y[5], x[5];
    for (int r = 0; r < 5; ++r) {
      rv[r] = r < C ? J.b[(size_t)r * K + k] : 0.0;
      P.r[(size_t)r * K + k] = rv[r];
      P.p[(size_t)r * K + k] = 0.0;
      J.lambda[(size_t)r * K + k] = 0.0;
    }
    for (int i = 0; i < C; ++i) {
      double s = rv[i];
      for (int q = 0; q < i; ++q) s -= D[pk5(i, q)] * y[q];
      y[i] = s / D[pk5(i, i)];
    }
    for (int i = C - 1; i >= 0; --i) {
      double s = y[i];
      for (int q = i + 1; q < C; ++q) s -= D[pk5(q, i)] * x[q];
      x[i] = s / D[pk5(i, i)];
    }
    for (int r = 0; r < 5; ++r) {
      const double zz = r < C ? x[r] : 0.0;
      P.z[(size_t)r * K + k] = zz;
      rz += rv[r] * zz;
      rr += rv[r] * rv[r];
    }
  }
  // block partial sums (fixed order: deterministic)
  __shared__ double s1[128], s2[128];
  s1[threadIdx.x] = rz;
  s2[threadIdx.x] = rr;
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    P.part[blockIdx.x] = s1[0];
    P.part[P.nblocks + blockIdx.x] = s2[0];
  }
}

// sums the per-block partials in a fixed order (one block)
__device__ __forceinline__ void block_sum2(const double *part, int n, int nb, double &a, double &b) {
  __shared__ double s1[PCG_THREADS], s2[PCG_THREADS];
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

__global__ void k_pcg_setup_reduce(DevPCG P, double rtol) {
  double rz, rr;
  block_sum2(P.part, P.nblocks, P.nblocks, rz, rr);
  if (threadIdx.x == 0) {
    P.scal[0] = rz;
    P.scal[2] = 0.0;      // beta of the first iteration
    P.scal[3] = rr;
    P.scal[4] = rr;       // |b|^2
    P.scal[5] = rtol * rtol;
    P.iter[0] = 0;
    P.iter[1] = (rr == 0.0) ? 1 : 0;
  }
}

// per body: zb_j = Hbar^{-1} sum_rows p_r W_r with p = z + beta p_old
template <bool XJ>
__global__ void __launch_bounds__(128) k_pcg_body(DevBodies B, DevJoints J, DevIncidence I, DevPCG P) {
  if (P.iter[1]) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= B.M || B.fixed[j]) return;
  const int K = J.K, M = B.M;
  const double beta = P.scal[2];
  double R[9], g[12];
  load_R(B.R, M, j, R);
#pragma unroll
  for (int a = 0; a < 12; ++a) g[a] = 0.0;
  for (int e = I.off[j]; e < I.off[j + 1]; ++e) {
    const int k = I.joint[e];
    double E[5][3], PR[5][3], WR[5];
    const int side = I.side[e];
    const int C = joint_rows_pt<double, XJ>(J, k, side, R, E, PR, WR);
    const int type = J.type[k];
    const bool full = J.qf && side == 0 && (type == 1 || (XJ && type == 3));
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      if (r >= C) break;
      const double pr = P.z[(size_t)r * K + k] + beta * P.p[(size_t)r * K + k];
      if (full) {  // MABD_JACOBIAN_FULL: the frame term on body a
        double qh[3];
        load_qf(J.qf, K, k, r, qh);
        add_skew_force(qh, pr, g);
      }
      const double *pp = PR[r];
      const double w = WR[r];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double v = pr * E[r][a];
        g[a] += pp[0] * v;
        g[3 + a] += pp[1] * v;
        g[6 + a] += pp[2] * v;
        g[9 + a] += w * v;
      }
    }
  }
  double h[16], z[12];
  load_hinv(B, j, h);
  hinv_apply(h, g, z);
#pragma unroll
  for (int a = 0; a < 12; ++a) P.zb[(size_t)a * M + j] = z[a];
}

// per joint: p = z + beta p_old (stored), Sp = sum_bodies W zb, partial p.Sp
template <bool XJ>
__global__ void __launch_bounds__(128) k_pcg_joint_sp(DevBodies B, DevJoints J, DevPCG P) {
  if (P.iter[1]) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int K = J.K;
  double psp = 0.0;
  if (k < K) {
    const int C = joint_nrows(J.type[k]);
    const uint8_t fl = J.flags[k];
    const double beta = P.scal[2];
    double pv[5], sp[5];
    for (int r = 0; r < 5; ++r) {
      pv[r] = r < C ? P.z[(size_t)r * K + k] + beta * P.p[(size_t)r * K + k] : 0.0;
      sp[r] = 0.0;
    }
    for (int side = 0; side < 2; ++side) {
      if (!(fl & (side == 0 ? JF_A_FREE : JF_B_FREE))) continue;
      const int j = side == 0 ? J.ja[k] : J.jb[k];
      double W[5][12], zb[12];
      joint_side_rows<XJ>(B, J, k, side, W);
      load12(P.zb, B.M, j, zb);
#pragma unroll
      for (int r = 0; r < 5; ++r) {
        if (r >= C) break;
        double v = 0.0;
#pragma unroll
        for (int a = 0; a < 12; ++a) v += W[r][a] * zb[a];
        sp[r] += v;
      }
    }
    for (int r = 0; r < 5; ++r) {
      P.p[(size_t)r * K + k] = pv[r];
      P.Sp[(size_t)r * K + k] = sp[r];
      psp += pv[r] * sp[r];
    }
  }
  __shared__ double s1[128];
  s1[threadIdx.x] = psp;
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (threadIdx.x < o) s1[threadIdx.x] += s1[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) P.part[blockIdx.x] = s1[0];
}

__global__ void k_pcg_alpha(DevPCG P) {
  if (P.iter[1]) return;
  double psp, dummy;
  block_sum2(P.part, P.nblocks, 0, psp, dummy);
  if (threadIdx.x == 0) {
    P.scal[6] = psp;
    P.scal[1] = psp > 0.0 ? P.scal[0] / psp : 0.0;
  }
}

// per joint: lambda += alpha p, r -= alpha Sp, z = D^{-1} r, partials r.z, r.r
__global__ void __launch_bounds__(128) k_pcg_joint_update(DevJoints J, DevPCG P) {
  if (P.iter[1]) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int K = J.K;
  double rz = 0.0, rr = 0.0;
  if (k < K) {
    const int C = joint_nrows(J.type[k]);
    const double alpha = P.scal[1];
    double rv[5], L[15], y[5], x[5];
    for (int r = 0; r < 5; ++r) {
      const size_t o = (size_t)r * K + k;
      J.lambda[o] += alpha * P.p[o];
      rv[r] = P.r[o] - alpha * P.Sp[o];
      P.r[o] = rv[r];
    }
#pragma unroll
    for (int i = 0; i < 15; ++i) L[i] = P.Lpre[(size_t)i * K + k];
    for (int i = 0; i < C; ++i) {
      double s = rv[i];
      for (int q = 0; q < i; ++q) s -= L[pk5(i, q)] * y[q];
      y[i] = s / L[pk5(i, i)];
    }
    for (int i = C - 1; i >= 0; --i) {
      double s = y[i];
      for (int q = i + 1; q < C; ++q) s -= L[pk5(q, i)] * x[q];
      x[i] = s / L[pk5(i, i)];
    }
    for (int r = 0; r < 5; ++r) {
      const double zz = r < C ? x[r] : 0.0;
      P.z[(size_t)r * K + k] = zz;
      rz += rv[r] * zz;
      rr += rv[r] * rv[r];
    }
  }
  __shared__ double s1[128], s2[128];
  s1[threadIdx.x] = rz;
  s2[threadIdx.x] = rr;
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    P.part[blockIdx.x] = s1[0];
    P.part[P.nblocks + blockIdx.x] = s2[0];
  }
}

__global__ void k_pcg_beta(DevPCG P, int max_iters) {
  if (P.iter[1]) return;
  double rz, rr;
  block_sum2(P.part, P.nblocks, P.nblocks, rz, rr);
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

void launch_pcg_setup(const DevBodies &B, const DevJoints &J, const DevPCG &P, double rtol,
                      int *status, cudaStream_t s) {
  if (J.xj) k_pcg_setup<true><<<P.nblocks, 128, 0, s>>>(B, J, P, status);
  else k_pcg_setup<false><<<P.nblocks, 128, 0, s>>>(B, J, P, status);
  k_pcg_setup_reduce<<<1, PCG_THREADS, 0, s>>>(P, rtol);
}

void launch_pcg_iteration(const DevBodies &B, const DevJoints &J, const DevIncidence &I,
                          const DevPCG &P, int max_iters, cudaStream_t s) {
  if (J.xj) {
    k_pcg_body<true><<<(B.M + 127) / 128, 128, 0, s>>>(B, J, I, P);
    k_pcg_joint_sp<true><<<P.nblocks, 128, 0, s>>>(B, J, P);
  } else {
    k_pcg_body<false><<<(B.M + 127) / 128, 128, 0, s>>>(B, J, I, P);
    k_pcg_joint_sp<false><<<P.nblocks, 128, 0, s>>>(B, J, P);
  }
  k_pcg_alpha<<<1, PCG_THREADS, 0, s>>>(P);
  k_pcg_joint_update<<<P.nblocks, 128, 0, s>>>(J, P);
  k_pcg_beta<<<1, PCG_THREADS, 0, s>>>(P, max_iters);
}

}  // namespace mabd
