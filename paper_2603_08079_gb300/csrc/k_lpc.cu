// Learned block preconditioner for the dual PCG: inference.
//
// Nodes are the (ball) joints, edges join joints that share a free body.  For
// the current state the dual S = G H^{-1} G^T (Eq. dual) is normalized by the
// inverse Cholesky factors C_k of its 3x3 diagonal blocks D_k, giving unit
// diagonal blocks and off-diagonal blocks E_kk' = C_k S_kk' C_k'^T.  A
// three-layer message-passing network (hidden width 64, each layer
// h' = relu([h_k, mean_{k'~k} h_k'] W + b), the products in BF16 on the tensor
// cores with FP32 accumulation) maps per-joint features of E to
//   s_k = exp(wd.h_k + cd)                                   (joint scale)
//   alpha_kk' = 1.5 sigmoid(a_k.b_k' + we0 |E_kk'| + we1 tr E_kk' + ce)
// for each edge to a lower-index neighbour k' < k (a = Wa^T h, b = Wb^T h),
// and the preconditioner is M^{-1} = C^T G^T G C with G = diag(s)(I - A),
// A_kk' = alpha_kk' E_kk'.  G is block lower triangular with diagonal blocks
// s_k I, so M^{-1} is symmetric positive definite for any parameters; with
// alpha = 0 and s = 1 it is block Jacobi.
#include <cuda_bf16.h>

#include "lpc_apply.cuh"
#include "mabd_f32.cuh"

namespace mabd {

__device__ __forceinline__ uint16_t f2bf(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf2f(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }

// ---------------------------------------------------------------------------
// normalized dual blocks
// ---------------------------------------------------------------------------
// joint point of joint k on its side `side` (FP32 copy)
__device__ __forceinline__ void jpoint(const DevJoints &J, int k, int side, float p[3]) {
  load3f(side == 0 ? J.pa1f : J.pb1f, J.K, k, p);
}

// world block R Mbar(p, q) R^T of body j
__device__ __forceinline__ void world_block(const DevBodies &B, int j, const float p[3], const float q[3],
                                            float out[9]) {
  float R[9], h[16], Mb[3][3], T[9];
  load_Rf(B, j, R);
  load_hf(B, j, h);
  mbar(h, p, q, Mb);
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) T[3 * r + c] = R[3 * r] * Mb[0][c] + R[3 * r + 1] * Mb[1][c] + R[3 * r + 2] * Mb[2][c];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) out[3 * r + c] = T[3 * r] * R[3 * c] + T[3 * r + 1] * R[3 * c + 1] + T[3 * r + 2] * R[3 * c + 2];
}

// per joint: D_k = sum over its free bodies of R Mbar(p, p) R^T, and
// C_k = L^{-1} for D_k = L L^T (packed lower: c00 c10 c11 c20 c21 c22)
__global__ void __launch_bounds__(128) k_lpc_chol(DevBodies B, DevJoints J, LpcGraph G, LpcAct A,
                                                  int *status) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= G.K) return;
  float D[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  const uint8_t fl = J.flags[k];
  for (int side = 0; side < 2; ++side) {
    if (!(fl & (side == 0 ? JF_A_FREE : JF_B_FREE))) continue;
    const int j = side == 0 ? J.ja[k] : J.jb[k];
    float p[3], blk[9];
    jpoint(J, k, side, p);
    world_block(B, j, p, p, blk);
#pragma unroll
    for (int i = 0; i < 9; ++i) D[i] += blk[i];
  }
  float l00 = D[0];
  if (!(l00 > 0.f)) {
    set_status(status, ST_NOT_SPD);
    l00 = 1.f;
  }
  l00 = sqrtf(l00);
  const float l10 = D[3] / l00, l20 = D[6] / l00;
  float l11 = D[4] - l10 * l10;
  if (!(l11 > 0.f)) {
    set_status(status, ST_NOT_SPD);
    l11 = 1.f;
  }
  l11 = sqrtf(l11);
  const float l21 = (D[7] - l20 * l10) / l11;
  float l22 = D[8] - l20 * l20 - l21 * l21;
  if (!(l22 > 0.f)) {
    set_status(status, ST_NOT_SPD);
    l22 = 1.f;
  }
  l22 = sqrtf(l22);
  // inverse of the lower factor
  const float c00 = 1.f / l00, c11 = 1.f / l11, c22 = 1.f / l22;
  const float c10 = -l10 * c00 * c11;
  const float c21 = -l21 * c11 * c22;
  const float c20 = -(l20 * c00 + l21 * c10) * c22;
  float *C = A.C + (size_t)6 * k;
  C[0] = c00; C[1] = c10; C[2] = c11; C[3] = c20; C[4] = c21; C[5] = c22;
}

__device__ __forceinline__ void unpackC(const float *Cp, float C[9]) {
  C[0] = Cp[0]; C[1] = 0.f;   C[2] = 0.f;
  C[3] = Cp[1]; C[4] = Cp[2]; C[5] = 0.f;
  C[6] = Cp[3]; C[7] = Cp[4]; C[8] = Cp[5];
}

// per joint k and each entry e (neighbour n through body j):
// S_kn = s_k s_n R_j Mbar_j(p_k, p_n) R_j^T, E_e = C_k S_kn C_n^T
__global__ void __launch_bounds__(128) k_lpc_edges(DevBodies B, DevJoints J, LpcGraph G, LpcAct A) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= G.K) return;
  float Ck[9];
  unpackC(A.C + (size_t)6 * k, Ck);
  for (int e = G.off[k]; e < G.off[k + 1]; ++e) {
    const int n = G.nbr[e], j = G.body[e];
    float pk_[3], pn[3], S[9], Cn[9], T[9];
    jpoint(J, k, G.sk[e], pk_);
    jpoint(J, n, G.sn[e], pn);
    world_block(B, j, pk_, pn, S);
    const float sg = (G.sk[e] == G.sn[e]) ? 1.f : -1.f;
    unpackC(A.C + (size_t)6 * n, Cn);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) T[3 * r + c] = Ck[3 * r] * S[c] + Ck[3 * r + 1] * S[3 + c] + Ck[3 * r + 2] * S[6 + c];
    float *Ee = A.E + (size_t)LPC_ES * e;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        Ee[3 * r + c] = sg * (T[3 * r] * Cn[3 * c] + T[3 * r + 1] * Cn[3 * c + 1] + T[3 * r + 2] * Cn[3 * c + 2]);
  }
}

void launch_lpc_blocks(const DevBodies &B, const DevJoints &J, const LpcGraph &G, const LpcAct &A,
                       int *status, cudaStream_t s) {
  if (G.K <= 0) return;
  const int nb = (G.K + 127) / 128;
  k_lpc_chol<<<nb, 128, 0, s>>>(B, J, G, A, status);
  k_lpc_edges<<<nb, 128, 0, s>>>(B, J, G, A);
}

// ---------------------------------------------------------------------------
// network
// ---------------------------------------------------------------------------
// features of joint k: 1, degree/8, lower degree/8, one-sided, sum |E|^2,
// max |E|, sum tr E, sum over lower neighbours |E|^2
__global__ void __launch_bounds__(128) k_lpc_features(LpcGraph G, LpcAct A) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= G.K) return;
  float f2 = 0.f, fmx = 0.f, ftr = 0.f, flo = 0.f;
  int lower = 0;
  for (int e = G.off[k]; e < G.off[k + 1]; ++e) {
    const float *Ee = A.E + (size_t)LPC_ES * e;
    float n2 = 0.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) n2 += Ee[i] * Ee[i];
    f2 += n2;
    fmx = fmaxf(fmx, sqrtf(n2));
    ftr += Ee[0] + Ee[4] + Ee[8];
    if (G.nbr[e] < k) {
      flo += n2;
      ++lower;
    }
  }
  float *x = A.x + (size_t)LPC_F * k;
  x[0] = 1.f;
  x[1] = (float)(G.off[k + 1] - G.off[k]) * 0.125f;
  x[2] = (float)lower * 0.125f;
  x[3] = G.onesided[k] ? 1.f : 0.f;
  x[4] = f2;
  x[5] = fmx;
  x[6] = ftr;
  x[7] = flo;
}

// bf16 transposed weights Wt[n][i] = W[i][n] of a layer with 2*KIN inputs
__global__ void k_lpc_wt(const float *P, uint16_t *W1t, uint16_t *W2t, uint16_t *W3t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  constexpr int N1 = 2 * LPC_F * LPC_H, N2 = 2 * LPC_H * LPC_H;
  if (i < N1) {
    const int n = i / (2 * LPC_F), r = i % (2 * LPC_F);
    W1t[i] = f2bf(P[LPC_OFF_W1 + r * LPC_H + n]);
  }
  if (i < N2) {
    const int n = i / (2 * LPC_H), r = i % (2 * LPC_H);
    W2t[i] = f2bf(P[LPC_OFF_W2 + r * LPC_H + n]);
    W3t[i] = f2bf(P[LPC_OFF_W3 + r * LPC_H + n]);
  }
}

void launch_lpc_weights(const float *P, uint16_t *W1t, uint16_t *W2t, uint16_t *W3t, cudaStream_t s) {
  k_lpc_wt<<<(2 * LPC_H * LPC_H + 255) / 256, 256, 0, s>>>(P, W1t, W2t, W3t);
}

// D (16x8 FP32) += A (16x16 BF16, row-major) x B (16x8 BF16, column-major)
__device__ __forceinline__ void mma_bf16(float d[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// One message-passing layer: per node the row [h_k, mean_{k'~k} h_k'] (2 KIN,
// rounded to BF16) times W (2 KIN x 64, BF16) on the tensor cores, FP32
// accumulation, + b, relu.  Each warp owns 16 nodes; the block stages W^T.
template <int KIN>
__global__ void __launch_bounds__(128) k_gnn_layer(LpcGraph G, const float *hin, const uint16_t *Wt,
                                                   const float *bias, float *Asave, float *pre,
                                                   float *hout) {
  constexpr int KA = 2 * KIN;
  __shared__ __align__(16) uint16_t Ws[LPC_H * KA];
  __shared__ __align__(16) uint16_t As[4][16 * KA];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < LPC_H * KA; i += blockDim.x) Ws[i] = Wt[i];
  const int row0 = (blockIdx.x * 4 + warp) * 16;
  uint16_t *Aw = As[warp];
  for (int idx = lane; idx < 16 * KIN; idx += 32) {
    const int i = idx / KIN, c = idx % KIN;
    const int node = row0 + i;
    float self = 0.f, mean = 0.f;
    if (node < G.K) {
      self = hin[(size_t)node * KIN + c];
      const int e0 = G.off[node], e1 = G.off[node + 1];
      float acc = 0.f;
      for (int e = e0; e < e1; ++e) acc += hin[(size_t)G.nbr[e] * KIN + c];
      mean = e1 > e0 ? acc / (float)(e1 - e0) : 0.f;
    }
    const uint16_t bs = f2bf(self), bm = f2bf(mean);
    Aw[i * KA + c] = bs;
    Aw[i * KA + KIN + c] = bm;
    if (Asave && node < G.K) {
      Asave[(size_t)node * KA + c] = bf2f(bs);
      Asave[(size_t)node * KA + KIN + c] = bf2f(bm);
    }
  }
  __syncthreads();
  const int g = lane >> 2, tig = lane & 3;
  float acc[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[nt][q] = 0.f;
#pragma unroll
  for (int ks = 0; ks < KA / 16; ++ks) {
    const int k0 = ks * 16 + tig * 2;
    const uint32_t a0 = *reinterpret_cast<const uint32_t *>(&Aw[g * KA + k0]);
    const uint32_t a1 = *reinterpret_cast<const uint32_t *>(&Aw[(g + 8) * KA + k0]);
    const uint32_t a2 = *reinterpret_cast<const uint32_t *>(&Aw[g * KA + k0 + 8]);
    const uint32_t a3 = *reinterpret_cast<const uint32_t *>(&Aw[(g + 8) * KA + k0 + 8]);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int n = nt * 8 + g;
      const uint32_t b0 = *reinterpret_cast<const uint32_t *>(&Ws[n * KA + k0]);
      const uint32_t b1 = *reinterpret_cast<const uint32_t *>(&Ws[n * KA + k0 + 8]);
      mma_bf16(acc[nt], a0, a1, a2, a3, b0, b1);
    }
  }
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
      const int node = row0 + g + 8 * rr;
      if (node >= G.K) continue;
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const int col = nt * 8 + tig * 2 + cc;
        const float v = acc[nt][2 * rr + cc] + bias[col];
        if (pre) pre[(size_t)node * LPC_H + col] = v;
        hout[(size_t)node * LPC_H + col] = fmaxf(v, 0.f);
      }
    }
}

// per joint: s = exp(wd.h + cd) (exponent clamped to [-8, 8]), a = Wa^T h, b = Wb^T h
__global__ void __launch_bounds__(128) k_lpc_head_node(LpcGraph G, LpcNet N, LpcAct A) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= G.K) return;
  const float *h = A.h3 + (size_t)LPC_H * k;
  const float *P = N.P;
  float d = P[LPC_OFF_CD], a[LPC_R], b[LPC_R];
#pragma unroll
  for (int r = 0; r < LPC_R; ++r) a[r] = b[r] = 0.f;
  for (int i = 0; i < LPC_H; ++i) {
    const float hi = h[i];
    d += P[LPC_OFF_WD + i] * hi;
#pragma unroll
    for (int r = 0; r < LPC_R; ++r) {
      a[r] += P[LPC_OFF_WA + i * LPC_R + r] * hi;
      b[r] += P[LPC_OFF_WB + i * LPC_R + r] * hi;
    }
  }
  A.s[k] = expf(fminf(fmaxf(d, -8.f), 8.f));
#pragma unroll
  for (int r = 0; r < LPC_R; ++r) {
    A.a[(size_t)LPC_R * k + r] = a[r];
    A.b[(size_t)LPC_R * k + r] = b[r];
  }
}

__device__ __forceinline__ void edge_feats(const float *Ee, float &nrm, float &tr) {
  float n2 = 0.f;
#pragma unroll
  for (int i = 0; i < 9; ++i) n2 += Ee[i] * Ee[i];
  nrm = sqrtf(n2);
  tr = Ee[0] + Ee[4] + Ee[8];
}

// per joint k, each entry e to a lower neighbour n: alpha_e; other entries 0
__global__ void __launch_bounds__(128) k_lpc_head_edge(LpcGraph G, LpcNet N, LpcAct A) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= G.K) return;
  const float *P = N.P;
  float a[LPC_R];
#pragma unroll
  for (int r = 0; r < LPC_R; ++r) a[r] = A.a[(size_t)LPC_R * k + r];
  for (int e = G.off[k]; e < G.off[k + 1]; ++e) {
    const int n = G.nbr[e];
    if (n >= k) {
      A.alpha[e] = 0.f;
      continue;
    }
    float nrm, tr;
    edge_feats(A.E + (size_t)LPC_ES * e, nrm, tr);
    float z = P[LPC_OFF_CE] + P[LPC_OFF_WE] * nrm + P[LPC_OFF_WE + 1] * tr;
#pragma unroll
    for (int r = 0; r < LPC_R; ++r) z += a[r] * A.b[(size_t)LPC_R * n + r];
    A.alpha[e] = 1.5f / (1.f + expf(-z));
  }
}

void launch_lpc_forward(const LpcGraph &G, const LpcNet &N, const LpcAct &A, bool keep, cudaStream_t s) {
  if (G.K <= 0) return;
  const int nb = (G.K + 127) / 128, nl = (G.K + 63) / 64;
  k_lpc_features<<<nb, 128, 0, s>>>(G, A);
  k_gnn_layer<LPC_F><<<nl, 128, 0, s>>>(G, A.x, N.W1t, N.P + LPC_OFF_B1, keep ? A.A1 : nullptr,
                                         keep ? A.pre1 : nullptr, A.h1);
  k_gnn_layer<LPC_H><<<nl, 128, 0, s>>>(G, A.h1, N.W2t, N.P + LPC_OFF_B2, keep ? A.A2 : nullptr,
                                         keep ? A.pre2 : nullptr, A.h2);
  k_gnn_layer<LPC_H><<<nl, 128, 0, s>>>(G, A.h2, N.W3t, N.P + LPC_OFF_B3, keep ? A.A3 : nullptr,
                                         keep ? A.pre3 : nullptr, A.h3);
  k_lpc_head_node<<<nb, 128, 0, s>>>(G, N, A);
  k_lpc_head_edge<<<nb, 128, 0, s>>>(G, N, A);
}

// ---------------------------------------------------------------------------
// preconditioner application inside the FP32 PCG ([5][K] vectors, rows 0-2)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_lpc_y(LpcGraph G, LpcAct A, const float *t, float *y,
                                               const int *iter) {
  if (iter && iter[1]) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < G.K) lpc_y_one(G, A, t, y, k);
}

// z = C^T G^T y and the per-block partial sums of r . z
__global__ void __launch_bounds__(128) k_lpc_z(LpcGraph G, LpcAct A, const float *y, const float *r,
                                               float *z, double *part, const int *iter) {
  if (iter && iter[1]) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const float rz = k < G.K ? lpc_z_one(G, A, y, r, z, k) : 0.f;
  __shared__ double s1[128];
  s1[threadIdx.x] = (double)rz;
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (threadIdx.x < o) s1[threadIdx.x] += s1[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s1[0];
}

void launch_lpc_apply(const LpcGraph &G, const LpcAct &A, const float *t, float *y, const float *r,
                      float *z, double *part, int nblocks, cudaStream_t s, const int *iter) {
  k_lpc_y<<<nblocks, 128, 0, s>>>(G, A, t, y, iter);
  k_lpc_z<<<nblocks, 128, 0, s>>>(G, A, y, r, z, part, iter);
}

}  // namespace mabd
