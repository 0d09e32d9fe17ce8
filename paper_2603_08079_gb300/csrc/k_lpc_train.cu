// Learned block preconditioner: training (forward in the inference kernels,
// backward and the optimizer here).
//
// Two objectives over a batch of normalized dual systems S~ (unit diagonal
// blocks, off-diagonal blocks E), X = G S~ G^T, G = diag(s)(I - A), n = 3K,
// estimated with probe vectors v (E[v v^T] = I):
//   Frobenius  L = sum_v |X v - v|^2 / (nv n);
//   Kaporin    L = log(tr X / n) - log det(X)^{1/n} + const
//              = log(sum_v v.X v / (nv n)) - (2/K) sum_k log s_k,
// the log of Kaporin's condition number (which bounds the CG iteration
// count); det G = prod s_k^3 because G is block lower triangular.  With
// t = s v, u = t - A^T t, w = S~ u, m = w - A w, y = s m the gradients are
//   q = s dL/dy,  dL/dw = q - A^T q,  dL/du = S~ dL/dw,  dL/dt = dL/du - A dL/du,
//   dL/ds_k = dL/dy_k . m_k + dL/dt_k . v_k (- 2/(K s_k), Kaporin),
// where dL/dy = 2 (y - v) / (nv n) (Frobenius) or v / sum_v v.y (Kaporin);
//   dL/dalpha_kn = -q_k^T E_kn w_n - t_k^T E_kn (dL/du)_n   (n < k),
// then through the heads and the three layers (the BF16 rounding of the layer
// inputs is passed straight through).  Probe vectors are drawn on the device
// with SplitMix64 (Steele, Lea and Flood, 2014) unless given.
#include <cuda_bf16.h>

#include "mabd_device.cuh"

namespace mabd {

// ---------------------------------------------------------------------------
// probe vectors
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  return x ^ (x >> 31);
}

// uniform on [-sqrt 3, sqrt 3) (unit variance) from the top 24 bits of
// SplitMix64(seed + i)
__global__ void k_lpc_probe(float *V, size_t n, uint64_t seed) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t r = splitmix64(seed + i);
  const float u = (float)(r >> 40) * (1.0f / 16777216.0f);
  V[i] = (2.0f * u - 1.0f) * 1.7320508f;
}

// ---------------------------------------------------------------------------
// loss and its gradient with respect to alpha and s
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mv3f(const float *E, const float *x, float y[3]) {
  y[0] = E[0] * x[0] + E[1] * x[1] + E[2] * x[2];
  y[1] = E[3] * x[0] + E[4] * x[1] + E[5] * x[2];
  y[2] = E[6] * x[0] + E[7] * x[1] + E[8] * x[2];
}

// out_k = in_k + sgn * sum over entries e of k with n < k (lower), n > k
// (upper) or all: coef_e E_e in_n, coef = alpha_e (lower), alpha_rev(e)
// (upper) or 1 (all); scale_n multiplies in_n when given
enum { LPC_LOWER = 0, LPC_UPPER = 1, LPC_ALL = 2 };

template <int WHICH>
__device__ __forceinline__ void spmv_row(const LpcGraph &G, const LpcAct &A, int k, const float *in,
                                         const float *scale_n, float sgn, int K, float out[3]) {
  const float *ik = in + (size_t)3 * k;
  out[0] = ik[0];
  out[1] = ik[1];
  out[2] = ik[2];
  for (int e = G.off[k]; e < G.off[k + 1]; ++e) {
    const int n = G.nbr[e];
    float c = 1.f;
    if (WHICH == LPC_LOWER) {
      if (n >= k) continue;
      c = A.alpha[e];
    } else if (WHICH == LPC_UPPER) {
      if (n <= k) continue;
      c = A.alpha[G.rev[e]];
    }
    if (scale_n) c *= scale_n[n];
    float y[3];
    mv3f(A.E + (size_t)LPC_ES * e, in + (size_t)3 * n, y);
    out[0] += sgn * c * y[0];
    out[1] += sgn * c * y[1];
    out[2] += sgn * c * y[2];
  }
}

// t = s v ; u = t - A^T t   (two passes over the probe vectors)
__global__ void __launch_bounds__(128) k_lpc_l1(LpcGraph G, LpcAct A, LpcTrainWork W) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int K = G.K;
  if (k >= K) return;
  for (int i = 0; i < W.nv; ++i) {
    const size_t o = ((size_t)i * K + k) * 3;
    for (int c = 0; c < 3; ++c) W.t[o + c] = A.s[k] * W.V[o + c];
  }
}

template <int WHICH>
__global__ void __launch_bounds__(128) k_lpc_spmv(LpcGraph G, LpcAct A, const float *in, float *out,
                                                  float sgn, int nv) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int K = G.K;
  if (k >= K) return;
  for (int i = 0; i < nv; ++i) {
    float y[3];
    spmv_row<WHICH>(G, A, k, in + (size_t)i * K * 3, nullptr, sgn, K, y);
    const size_t o = ((size_t)i * K + k) * 3;
    out[o] = y[0];
    out[o + 1] = y[1];
    out[o + 2] = y[2];
  }
}

// pass 1: m = w - A w, y = s m; per block the sum of |y - v|^2 (Frobenius
// objective) or of v.y (Kaporin objective) into part[b], and of log s_k into
// part[nb + b]
__device__ __forceinline__ void block_sum2d(double a, double b, double *part, int nb) {
  __shared__ double sh[128], sh2[128];
  sh[threadIdx.x] = a;
  sh2[threadIdx.x] = b;
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sh[threadIdx.x] += sh[threadIdx.x + o];
      sh2[threadIdx.x] += sh2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x] = sh[0];
    part[nb + blockIdx.x] = sh2[0];
  }
}

__global__ void __launch_bounds__(128) k_lpc_l4a(LpcGraph G, LpcAct A, LpcTrainWork W, int kind) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int K = G.K;
  double acc = 0.0, lsum = 0.0;
  if (k < K) {
    const float sk = A.s[k];
    lsum = log((double)sk);
    for (int i = 0; i < W.nv; ++i) {
      float m[3];
      spmv_row<LPC_LOWER>(G, A, k, W.w + (size_t)i * K * 3, nullptr, -1.f, K, m);
      const size_t o = ((size_t)i * K + k) * 3;
      for (int c = 0; c < 3; ++c) {
        const double y = (double)(sk * m[c]), v = (double)W.V[o + c];
        acc += kind == 0 ? (y - v) * (y - v) : v * y;
      }
    }
  }
  block_sum2d(acc, lsum, W.part, gridDim.x);
}

// pass 2 (gradient): dL/dy = 2 (y - v) / N (Frobenius) or v / sum(v.y)
// (Kaporin, from loss[0]); q = s dL/dy, ds = dL/dy . m (- 2 / (K s) for
// Kaporin's determinant term), dalpha = -q_k^T E w_n
__global__ void __launch_bounds__(128) k_lpc_l4b(LpcGraph G, LpcAct A, LpcTrainWork W, int kind,
                                                 float cscale) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int K = G.K;
  if (k >= K) return;
  const float sk = A.s[k];
  const float ck = kind == 0 ? cscale : (float)(1.0 / W.loss[0]);
  float ds = kind == 0 ? 0.f : -2.f / ((float)K * sk);
  for (int e = G.off[k]; e < G.off[k + 1]; ++e)
    if (G.nbr[e] < k) W.dalpha[e] = 0.f;
  for (int i = 0; i < W.nv; ++i) {
    const float *wi = W.w + (size_t)i * K * 3;
    float m[3];
    spmv_row<LPC_LOWER>(G, A, k, wi, nullptr, -1.f, K, m);
    const size_t o = ((size_t)i * K + k) * 3;
    float q[3];
    for (int c = 0; c < 3; ++c) {
      const float gy = kind == 0 ? ck * (sk * m[c] - W.V[o + c]) : ck * W.V[o + c];
      ds += gy * m[c];
      q[c] = sk * gy;
      W.q[o + c] = q[c];
    }
    for (int e = G.off[k]; e < G.off[k + 1]; ++e) {
      const int n = G.nbr[e];
      if (n >= k) continue;
      float y[3];
      mv3f(A.E + (size_t)LPC_ES * e, wi + (size_t)3 * n, y);
      W.dalpha[e] -= q[0] * y[0] + q[1] * y[1] + q[2] * y[2];
    }
  }
  W.ds[k] = ds;
}

// dL/dt = gu - A gu; ds += dL/dt . v; dalpha -= t_k^T E gu_n
__global__ void __launch_bounds__(128) k_lpc_l7(LpcGraph G, LpcAct A, LpcTrainWork W) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int K = G.K;
  if (k >= K) return;
  float ds = W.ds[k];
  for (int i = 0; i < W.nv; ++i) {
    const float *gui = W.gu + (size_t)i * K * 3;
    float gt[3];
    spmv_row<LPC_LOWER>(G, A, k, gui, nullptr, -1.f, K, gt);
    const size_t o = ((size_t)i * K + k) * 3;
    ds += gt[0] * W.V[o] + gt[1] * W.V[o + 1] + gt[2] * W.V[o + 2];
    const float *tk = W.t + o;
    for (int e = G.off[k]; e < G.off[k + 1]; ++e) {
      const int n = G.nbr[e];
      if (n >= k) continue;
      float y[3];
      mv3f(A.E + (size_t)LPC_ES * e, gui + (size_t)3 * n, y);
      W.dalpha[e] -= tk[0] * y[0] + tk[1] * y[1] + tk[2] * y[2];
    }
  }
  W.ds[k] = ds;
}

// loss[0] = sum of part[0..n), loss[1] = sum of part[n..2n)
__global__ void k_lpc_loss_sum(const double *part, int n, double *loss) {
  __shared__ double sh[256], sh2[256];
  double x = 0.0, y = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    x += part[i];
    y += part[n + i];
  }
  sh[threadIdx.x] = x;
  sh2[threadIdx.x] = y;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sh[threadIdx.x] += sh[threadIdx.x + o];
      sh2[threadIdx.x] += sh2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    loss[0] = sh[0];
    loss[1] = sh2[0];
  }
}

// ---------------------------------------------------------------------------
// heads backward
// ---------------------------------------------------------------------------
// per joint: dz_e = dalpha_e alpha_e (1 - alpha_e / 1.5) for its lower entries
// (kept in dalpha), da_k = sum dz_e b_n, db_k = sum over upper entries of
// dz_rev a_n, dd_k = ds_k s_k (0 where the exponent was clamped), then
// dh3_k = Wa da + Wb db + wd dd and the head parameter gradients
__global__ void __launch_bounds__(128) k_lpc_head_dz(LpcGraph G, LpcAct A, LpcTrainWork W) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= G.K) return;
  for (int e = G.off[k]; e < G.off[k + 1]; ++e) {
    if (G.nbr[e] >= k) continue;
    const float al = A.alpha[e];
    W.dalpha[e] *= al * (1.f - al * (1.f / 1.5f));
  }
}

__global__ void __launch_bounds__(128) k_lpc_head_bwd(LpcGraph G, LpcAct A, LpcNet N, LpcTrainWork W) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const float *P = N.P;
  __shared__ float gWa[LPC_H * LPC_R], gWb[LPC_H * LPC_R], gwd[LPC_H], gsc[4];
  for (int i = threadIdx.x; i < LPC_H * LPC_R; i += blockDim.x) gWa[i] = gWb[i] = 0.f;
  for (int i = threadIdx.x; i < LPC_H; i += blockDim.x) gwd[i] = 0.f;
  if (threadIdx.x < 4) gsc[threadIdx.x] = 0.f;
  __syncthreads();
  if (k < G.K) {
    float da[LPC_R], db[LPC_R];
#pragma unroll
    for (int r = 0; r < LPC_R; ++r) da[r] = db[r] = 0.f;
    float gwe0 = 0.f, gwe1 = 0.f, gce = 0.f;
    for (int e = G.off[k]; e < G.off[k + 1]; ++e) {
      const int n = G.nbr[e];
      if (n < k) {
        const float dz = W.dalpha[e];
#pragma unroll
        for (int r = 0; r < LPC_R; ++r) da[r] += dz * A.b[(size_t)LPC_R * n + r];
        const float *Ee = A.E + (size_t)LPC_ES * e;
        float n2 = 0.f;
#pragma unroll
        for (int i = 0; i < 9; ++i) n2 += Ee[i] * Ee[i];
        gwe0 += dz * sqrtf(n2);
        gwe1 += dz * (Ee[0] + Ee[4] + Ee[8]);
        gce += dz;
      } else {
        const float dz = W.dalpha[G.rev[e]];
#pragma unroll
        for (int r = 0; r < LPC_R; ++r) db[r] += dz * A.a[(size_t)LPC_R * n + r];
      }
    }
    // exponent of s before clamping
    float d = P[LPC_OFF_CD];
    const float *h = A.h3 + (size_t)LPC_H * k;
    for (int i = 0; i < LPC_H; ++i) d += P[LPC_OFF_WD + i] * h[i];
    const float dd = (d > -8.f && d < 8.f) ? W.ds[k] * A.s[k] : 0.f;
    float *dh = W.dh + (size_t)LPC_H * k;
    for (int i = 0; i < LPC_H; ++i) {
      float v = P[LPC_OFF_WD + i] * dd;
#pragma unroll
      for (int r = 0; r < LPC_R; ++r) v += P[LPC_OFF_WA + i * LPC_R + r] * da[r] + P[LPC_OFF_WB + i * LPC_R + r] * db[r];
      dh[i] = v;
      const float hi = h[i];
      if (hi != 0.f) {
        atomicAdd(&gwd[i], hi * dd);
#pragma unroll
        for (int r = 0; r < LPC_R; ++r) {
          atomicAdd(&gWa[i * LPC_R + r], hi * da[r]);
          atomicAdd(&gWb[i * LPC_R + r], hi * db[r]);
        }
      }
    }
    atomicAdd(&gsc[0], dd);
    atomicAdd(&gsc[1], gwe0);
    atomicAdd(&gsc[2], gwe1);
    atomicAdd(&gsc[3], gce);
  }
  __syncthreads();
  float *g = W.grad;
  for (int i = threadIdx.x; i < LPC_H * LPC_R; i += blockDim.x) {
    atomicAdd(&g[LPC_OFF_WA + i], gWa[i]);
    atomicAdd(&g[LPC_OFF_WB + i], gWb[i]);
  }
  for (int i = threadIdx.x; i < LPC_H; i += blockDim.x) atomicAdd(&g[LPC_OFF_WD + i], gwd[i]);
  if (threadIdx.x == 0) {
    atomicAdd(&g[LPC_OFF_CD], gsc[0]);
    atomicAdd(&g[LPC_OFF_WE], gsc[1]);
    atomicAdd(&g[LPC_OFF_WE + 1], gsc[2]);
    atomicAdd(&g[LPC_OFF_CE], gsc[3]);
  }
}

// ---------------------------------------------------------------------------
// layer backward (FP32)
// ---------------------------------------------------------------------------
// per node: dpre = dh (pre > 0), dA = dpre W^T (W: the BF16 weights used forward)
template <int KIN>
__global__ void __launch_bounds__(128) k_gnn_bwd_a(int K, const float *dh, const float *pre,
                                                   const uint16_t *Wt, float *dpre, float *dA) {
  constexpr int KA = 2 * KIN;
  __shared__ float Ws[LPC_H * KA];  // [n][i]
  for (int i = threadIdx.x; i < LPC_H * KA; i += blockDim.x)
    Ws[i] = __bfloat162float(__ushort_as_bfloat16(Wt[i]));
  __syncthreads();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  float dp[LPC_H];
  for (int n = 0; n < LPC_H; ++n) {
    const float v = pre[(size_t)k * LPC_H + n] > 0.f ? dh[(size_t)k * LPC_H + n] : 0.f;
    dp[n] = v;
    dpre[(size_t)k * LPC_H + n] = v;
  }
  for (int i = 0; i < KA; ++i) {
    float v = 0.f;
    for (int n = 0; n < LPC_H; ++n) v += dp[n] * Ws[n * KA + i];
    dA[(size_t)k * KA + i] = v;
  }
}

// dW[i][n] += sum_k A_k[i] dpre_k[n], db[n] += sum_k dpre_k[n]: block j covers
// a range of nodes; each thread owns weight entries, the block adds to grad
template <int KIN>
__global__ void __launch_bounds__(256) k_gnn_bwd_w(int K, const float *Asave, const float *dpre,
                                                   float *gW, float *gb, int rows_per_block) {
  constexpr int KA = 2 * KIN;
  const int r0 = blockIdx.x * rows_per_block, r1 = min(K, r0 + rows_per_block);
  for (int idx = threadIdx.x; idx < KA * LPC_H + LPC_H; idx += blockDim.x) {
    float acc = 0.f;
    if (idx < KA * LPC_H) {
      const int i = idx / LPC_H, n = idx % LPC_H;
      for (int k = r0; k < r1; ++k) acc += Asave[(size_t)k * KA + i] * dpre[(size_t)k * LPC_H + n];
      atomicAdd(&gW[idx], acc);
    } else {
      const int n = idx - KA * LPC_H;
      for (int k = r0; k < r1; ++k) acc += dpre[(size_t)k * LPC_H + n];
      atomicAdd(&gb[n], acc);
    }
  }
}

// dh_in_k = dA_k[0:KIN] + sum_{n ~ k} dA_n[KIN:2KIN] / deg(n)
template <int KIN>
__global__ void __launch_bounds__(128) k_gnn_bwd_h(LpcGraph G, const float *dA, float *dhin) {
  constexpr int KA = 2 * KIN;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= G.K) return;
  for (int c = 0; c < KIN; ++c) {
    float v = dA[(size_t)k * KA + c];
    for (int e = G.off[k]; e < G.off[k + 1]; ++e) {
      const int n = G.nbr[e];
      const int dn = G.off[n + 1] - G.off[n];
      v += dA[(size_t)n * KA + KIN + c] / (float)dn;
    }
    dhin[(size_t)k * KIN + c] = v;
  }
}

// ---------------------------------------------------------------------------
// Adam (Kingma and Ba, 2015)
// ---------------------------------------------------------------------------
__global__ void k_lpc_adam(float *P, const float *g, float *m, float *v, int n, float lr, float b1,
                           float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ---------------------------------------------------------------------------
// host-side launch sequences
// ---------------------------------------------------------------------------
void launch_lpc_probe(float *V, size_t n, uint64_t seed, cudaStream_t s) {
  if (n) k_lpc_probe<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(V, n, seed);
}

// loss of the batch (W.loss) and, when grad, the gradient of every
// parameter (W.grad, zeroed here); the forward pass must have run with keep
void launch_lpc_loss_grad(const LpcGraph &G, const LpcAct &A, const LpcNet &N, const LpcTrainWork &W,
                          int kind, bool grad, cudaStream_t s) {
  const int K = G.K, nb = (K + 127) / 128;
  const float cscale = 2.f / (float)(W.nv * 3 * (size_t)K);
  k_lpc_l1<<<nb, 128, 0, s>>>(G, A, W);
  k_lpc_spmv<LPC_UPPER><<<nb, 128, 0, s>>>(G, A, W.t, W.u, -1.f, W.nv);
  k_lpc_spmv<LPC_ALL><<<nb, 128, 0, s>>>(G, A, W.u, W.w, 1.f, W.nv);
  k_lpc_l4a<<<nb, 128, 0, s>>>(G, A, W, kind);
  k_lpc_loss_sum<<<1, 256, 0, s>>>(W.part, nb, W.loss);
  if (!grad) return;
  k_lpc_l4b<<<nb, 128, 0, s>>>(G, A, W, kind, cscale);
  cudaMemsetAsync(W.grad, 0, sizeof(float) * LPC_NPARAM, s);
  k_lpc_spmv<LPC_UPPER><<<nb, 128, 0, s>>>(G, A, W.q, W.gw, -1.f, W.nv);
  k_lpc_spmv<LPC_ALL><<<nb, 128, 0, s>>>(G, A, W.gw, W.gu, 1.f, W.nv);
  k_lpc_l7<<<nb, 128, 0, s>>>(G, A, W);
  k_lpc_head_dz<<<nb, 128, 0, s>>>(G, A, W);
  k_lpc_head_bwd<<<nb, 128, 0, s>>>(G, A, N, W);
  const int rpb = 256, nbw = (K + rpb - 1) / rpb;
  // layer 3
  k_gnn_bwd_a<LPC_H><<<nb, 128, 0, s>>>(K, W.dh, A.pre3, N.W3t, W.dpre, W.dA);
  k_gnn_bwd_w<LPC_H><<<nbw, 256, 0, s>>>(K, A.A3, W.dpre, W.grad + LPC_OFF_W3, W.grad + LPC_OFF_B3, rpb);
  k_gnn_bwd_h<LPC_H><<<nb, 128, 0, s>>>(G, W.dA, W.dh2);
  // layer 2
  k_gnn_bwd_a<LPC_H><<<nb, 128, 0, s>>>(K, W.dh2, A.pre2, N.W2t, W.dpre, W.dA);
  k_gnn_bwd_w<LPC_H><<<nbw, 256, 0, s>>>(K, A.A2, W.dpre, W.grad + LPC_OFF_W2, W.grad + LPC_OFF_B2, rpb);
  k_gnn_bwd_h<LPC_H><<<nb, 128, 0, s>>>(G, W.dA, W.dh);
  // layer 1 (no gradient with respect to the features)
  k_gnn_bwd_a<LPC_F><<<nb, 128, 0, s>>>(K, W.dh, A.pre1, N.W1t, W.dpre, W.dA);
  k_gnn_bwd_w<LPC_F><<<nbw, 256, 0, s>>>(K, A.A1, W.dpre, W.grad + LPC_OFF_W1, W.grad + LPC_OFF_B1, rpb);
}

void launch_lpc_adam(float *P, const float *g, float *m, float *v, float lr, int step, cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_lpc_adam<<<(LPC_NPARAM + 255) / 256, 256, 0, s>>>(P, g, m, v, LPC_NPARAM, lr, b1, b2, 1e-8f, c1, c2);
}

}  // namespace mabd
