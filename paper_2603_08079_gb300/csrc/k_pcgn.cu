// FP32 PCG of the mixed form on ball-joint graphs in the normalized dual
// space, as one cooperative launch per solve.
//
// With C_k the inverse Cholesky factor of the diagonal block D_k of
// S = G H^{-1} G^T (Eq. dual), the normalized dual S~ = C S C^T has identity
// diagonal blocks and the off-diagonal blocks E_kk' = C_k S_kk' C_k'^T that
// the learned preconditioner already forms each step (k_lpc.cu).  Solving
// S x = b is solving S~ x~ = C b with x = C^T x~, and the learned
// preconditioner C^T G^T G C of S is G^T G for S~ (block Jacobi: the
// identity).  So an iteration is one pass over the 3x3 blocks E (q = S~ p),
// then the residual update fused with y = G r (lower neighbours), then
// z = G^T y (upper neighbours): three phases, each a grid-stride loop over
// the joints, separated by the bounded grid barrier; the per-body matrix-free
// S-apply of k_pcg32.cu is not needed.  The stopping test is the one of
// k_pcg32.cu, |r| <= rtol |b| on the unnormalized residual r = C^{-1} r~.
// Vectors are one float4 per joint (three rows and a pad).
#include "grid_sync.cuh"
#include "mabd_f32.cuh"

namespace mabd {

__device__ __forceinline__ float3 ld3(const float4 *v, int k) {
  const float4 a = v[k];
  return make_float3(a.x, a.y, a.z);
}
__device__ __forceinline__ void st3(float4 *v, int k, float3 a) { v[k] = make_float4(a.x, a.y, a.z, 0.f); }
__device__ __forceinline__ float3 axpy3(float a, float3 x, float3 y) {
  return make_float3(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z));
}
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// E w for a stored block (row-major 3x3 in LPC_ES = 12 floats: three 16-byte loads)
__device__ __forceinline__ float3 emul(const float *E, float3 w) {
  const float4 a = *reinterpret_cast<const float4 *>(E), b = *reinterpret_cast<const float4 *>(E + 4),
               c = *reinterpret_cast<const float4 *>(E + 8);
  return make_float3(a.x * w.x + a.y * w.y + a.z * w.z, a.w * w.x + b.x * w.y + b.y * w.z,
                     b.z * w.x + b.w * w.y + c.x * w.z);
}

// C r with C packed lower (c00 c10 c11 c20 c21 c22)
__device__ __forceinline__ float3 cmul(const float *Cp, float3 r) {
  return make_float3(Cp[0] * r.x, Cp[1] * r.x + Cp[2] * r.y, Cp[3] * r.x + Cp[4] * r.y + Cp[5] * r.z);
}
// C^T x
__device__ __forceinline__ float3 ctmul(const float *Cp, float3 x) {
  return make_float3(Cp[0] * x.x + Cp[1] * x.y + Cp[3] * x.z, Cp[2] * x.y + Cp[4] * x.z, Cp[5] * x.z);
}
// C^{-T} l (back substitution with C^T)
__device__ __forceinline__ float3 ctinv(const float *Cp, float3 l) {
  const float x2 = l.z / Cp[5];
  const float x1 = (l.y - Cp[4] * x2) / Cp[2];
  const float x0 = (l.x - Cp[1] * x1 - Cp[3] * x2) / Cp[0];
  return make_float3(x0, x1, x2);
}
// C^{-1} t (forward substitution)
__device__ __forceinline__ float3 cinv(const float *Cp, float3 t) {
  const float r0 = t.x / Cp[0];
  const float r1 = (t.y - Cp[1] * r0) / Cp[2];
  const float r2 = (t.z - Cp[3] * r0 - Cp[4] * r1) / Cp[5];
  return make_float3(r0, r1, r2);
}

// The rows below walk a joint's neighbour list EU entries at a time, the
// loads of the EU issued together: one entry at a time, each gather waited
// for the previous entry's arithmetic, and the phase was a chain of memory
// round trips.
constexpr int EU = 4;

// neighbour of entry e; a MABD_DEBUG build treats one out of range as absent
// (the solve's first pass has already flagged it in the status word)
__device__ __forceinline__ int nbr_at(const LpcGraph &G, int e) {
  const int n = G.nbr[e];
#ifdef MABD_DEBUG
  if (n < 0 || n >= G.K) return -1;
#endif
  return n;
}

// q_k = p_k + sum_e E_e p_n with p = z + beta p_old formed on the fly
__device__ __forceinline__ float3 sapply_row(const LpcGraph &G, const LpcAct &A, const float4 *z, const float4 *po,
                                             float beta, int k, float3 pk) {
  float3 q = pk;
  const int e0 = G.off[k], e1 = G.off[k + 1];
  for (int e = e0; e < e1; e += EU) {
    int n[EU];
    float3 w[EU];
#pragma unroll
    for (int u = 0; u < EU; ++u) n[u] = e + u < e1 ? nbr_at(G, e + u) : -1;
#pragma unroll
    for (int u = 0; u < EU; ++u)
      w[u] = n[u] >= 0 ? axpy3(beta, ld3(po, n[u]), ld3(z, n[u])) : make_float3(0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < EU; ++u) {
      if (n[u] < 0) continue;
      const float3 t = emul(A.E + (size_t)LPC_ES * (e + u), w[u]);
      q.x += t.x;
      q.y += t.y;
      q.z += t.z;
    }
  }
  return q;
}

// y_k = s_k (r'_k - sum_{lower e} alpha_e E_e r'_n), r' = r - a q formed on the fly
__device__ __forceinline__ float3 lower_row(const LpcGraph &G, const LpcAct &A, const float4 *r, const float4 *q,
                                            float a, int k, float3 rk) {
  float3 v = rk;
  const int e0 = G.off[k], e1 = G.off[k + 1];
  for (int e = e0; e < e1; e += EU) {
    int n[EU];
    float3 w[EU];
#pragma unroll
    for (int u = 0; u < EU; ++u) {
      n[u] = e + u < e1 ? nbr_at(G, e + u) : -1;
      if (n[u] >= k) n[u] = -1;  // lower neighbours only
    }
#pragma unroll
    for (int u = 0; u < EU; ++u)
      w[u] = n[u] >= 0 ? axpy3(-a, ld3(q, n[u]), ld3(r, n[u])) : make_float3(0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < EU; ++u) {
      if (n[u] < 0) continue;
      const float3 t = emul(A.E + (size_t)LPC_ES * (e + u), w[u]);
      const float al = A.alpha[e + u];
      v.x -= al * t.x;
      v.y -= al * t.y;
      v.z -= al * t.z;
    }
    if (n[EU - 1] < 0) break;  // sorted by index: past the lower neighbours
  }
  const float sk = A.s[k];
  return make_float3(sk * v.x, sk * v.y, sk * v.z);
}

// z_k = s_k y_k - sum_{upper e} cu_e E_e y_n with cu_e = alpha_rev(e) s_n
// (formed once per solve)
__device__ __forceinline__ float3 upper_row(const LpcGraph &G, const LpcAct &A, const float *cu, const float4 *y,
                                            int k) {
  const float sk = A.s[k];
  const float3 yk = ld3(y, k);
  float3 u3 = make_float3(sk * yk.x, sk * yk.y, sk * yk.z);
  const int e0 = G.off[k], e1 = G.off[k + 1];
  for (int e = e1 - 1; e >= e0; e -= EU) {
    int n[EU];
    float3 w[EU];
    float al[EU];
#pragma unroll
    for (int u = 0; u < EU; ++u) {
      n[u] = e - u >= e0 ? nbr_at(G, e - u) : -1;
      if (n[u] <= k) n[u] = -1;  // upper neighbours only
    }
#pragma unroll
    for (int u = 0; u < EU; ++u) {
      w[u] = n[u] >= 0 ? ld3(y, n[u]) : make_float3(0.f, 0.f, 0.f);
      al[u] = n[u] >= 0 ? cu[e - u] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < EU; ++u) {
      if (n[u] < 0) continue;
      const float3 t = emul(A.E + (size_t)LPC_ES * (e - u), w[u]);
      u3.x -= al[u] * t.x;
      u3.y -= al[u] * t.y;
      u3.z -= al[u] * t.z;
    }
    if (n[EU - 1] < 0) break;  // sorted by index: past the upper neighbours
  }
  return u3;
}

// The whole solve (setup, iterations, x = C^T x~ out) in one cooperative
// launch, from x0 when given (the previous step's multipliers: a warm
// start; non-finite entries start at 0), else from 0.  LPC: the learned
// preconditioner; else block Jacobi (z = r~).
// One block of PN_THREADS per SM: on the 64x64x16 net that is one joint per
// thread (no thread of a phase carries a second joint), and a grid barrier
// or a grid sum has one arrival or one partial per SM.
constexpr int PN_THREADS = 896;

template <bool LPC>
__global__ void __launch_bounds__(PN_THREADS, 1)
    k_pcgn(LpcGraph G, LpcAct A, DevPCGN V, DevPCG32 P, const double *rhs, const double *x0, double rtol,
           int max_iters, double *out, double *acc, int *status) {
  __shared__ float sh[PN_THREADS];
  const unsigned nblk = gridDim.x;
  const int tid = blockIdx.x * PN_THREADS + threadIdx.x, nth = nblk * PN_THREADS;
  const int K = G.K;
#ifdef MABD_DEBUG
  // the joint graph once per solve: every neighbour and reverse entry in range
  for (int e = tid; e < G.nnz; e += nth)
    if (!MABD_INDEX_OK(G.nbr[e], K, status) || !MABD_INDEX_OK(G.rev[e], G.nnz, status)) break;
#endif
  // the scalar reductions in FP32 (the vectors are FP32; FP64 arithmetic is
  // the slow pipe here); fixed order, so every block gets the same sums
  float *fp = reinterpret_cast<float *>(P.ppart);
  float *prz = fp, *prr = fp + P32_MAXB, *ppq = fp + 2 * P32_MAXB, *pbb = fp + 3 * P32_MAXB;
  unsigned gen = 0;
  bool ok = true;
  int cur = 0, pc = 0;
  // setup: r~ = C b - S~ x~0 with x~0 = C^{-T} x0 (x0 = 0 when not given),
  // p_old = 0, z = M~^{-1} r~
  float bb = 0.f;
  {
    float rr = 0.f, rz = 0.f, rb = 0.f;
    for (int k = tid; k < K; k += nth) {
      const float3 b = make_float3((float)rhs[k], (float)rhs[(size_t)K + k], (float)rhs[2 * (size_t)K + k]);
      const float3 t = cmul(A.C + (size_t)6 * k, b);
      float3 xt = make_float3(0.f, 0.f, 0.f);
      if (x0) {
        const float3 l0 = make_float3((float)x0[k], (float)x0[(size_t)K + k], (float)x0[2 * (size_t)K + k]);
        if (isfinite(l0.x) && isfinite(l0.y) && isfinite(l0.z)) xt = ctinv(A.C + (size_t)6 * k, l0);
      }
      st3(V.r[0], k, t);
      st3(V.x, k, xt);
      st3(V.p[0], k, make_float3(0.f, 0.f, 0.f));
      st3(V.q, k, make_float3(0.f, 0.f, 0.f));
      rb += dot3(b, b);
      if (!x0) {
        rr += dot3(b, b);
        if (!LPC) {
          st3(V.z, k, t);
          rz += dot3(t, t);
        }
      }
    }
    if (x0) {
      // r~ = C b - (x~0 + sum_e E_e x~0_n): needs every joint's x~0
      ok = ok && grid_barrier(P.bar, nblk, gen);
      for (int k = tid; ok && k < K; k += nth) {
        const float3 xk = ld3(V.x, k);
        const float3 sx = sapply_row(G, A, V.x, V.p[0], 0.f, k, xk);
        const float3 t = ld3(V.r[0], k);
        const float3 r0 = make_float3(t.x - sx.x, t.y - sx.y, t.z - sx.z);
        st3(V.r[0], k, r0);
        const float3 ru = cinv(A.C + (size_t)6 * k, r0);
        rr += dot3(ru, ru);
        if (!LPC) {
          st3(V.z, k, r0);
          rz += dot3(r0, r0);
        }
      }
    }
    if (LPC) {
      for (int e = tid; e < G.nnz; e += nth) {
        const int n = nbr_at(G, e), r = G.rev[e];
        V.cu[e] = (n >= 0 && r >= 0 && r < G.nnz) ? A.alpha[r] * A.s[n] : 0.f;
      }
      ok = ok && grid_barrier(P.bar, nblk, gen);
      for (int k = tid; ok && k < K; k += nth) st3(V.y, k, lower_row(G, A, V.r[0], V.q, 0.f, k, ld3(V.r[0], k)));
      ok = ok && grid_barrier(P.bar, nblk, gen);
      for (int k = tid; ok && k < K; k += nth) {
        const float3 z = upper_row(G, A, V.cu, V.y, k);
        st3(V.z, k, z);
        rz += dot3(ld3(V.r[0], k), z);
      }
    }
    float bs[3] = {rz, rr, rb};
    block_sums<3, float, PN_THREADS>(bs, sh);
    if (threadIdx.x == 0) {
      prz[blockIdx.x] = bs[0];
      prr[blockIdx.x] = bs[1];
      pbb[blockIdx.x] = bs[2];
    }
    ok = ok && grid_barrier(P.bar, nblk, gen);
  }
  float gs[2];
  grid_sums<2, float, PN_THREADS>(fp, P32_MAXB, nblk, gs, sh);
  float rz = gs[0], rr = gs[1];
  bb = grid_sum<float, PN_THREADS>(pbb, nblk, sh);
  const float tol2 = (float)(rtol * rtol);
  float beta = 0.f;
  int it = 0;
  bool done = rr <= tol2 * bb;
  while (ok && !done && it < max_iters) {
    // A: p = z + beta p_old, q = S~ p, p.q
    float pq = 0.f;
    for (int k = tid; k < K; k += nth) {
      const float3 pk = axpy3(beta, ld3(V.p[pc], k), ld3(V.z, k));
      st3(V.p[pc ^ 1], k, pk);
      const float3 q = sapply_row(G, A, V.z, V.p[pc], beta, k, pk);
      st3(V.q, k, q);
      pq += dot3(pk, q);
    }
    const float bpq = block_sum<float, PN_THREADS>(pq, sh);
    if (threadIdx.x == 0) ppq[blockIdx.x] = bpq;
    ok = grid_barrier(P.bar, nblk, gen);
    if (!ok) break;
    const float pSp = grid_sum<float, PN_THREADS>(ppq, nblk, sh);
    const float a = pSp > 0.f ? rz / pSp : 0.f;
    // B: r' = r - a q, x += a p, |C^{-1} r'|^2; y = G r' (learned) or z = r'
    float rrf = 0.f, rzf = 0.f;
    for (int k = tid; k < K; k += nth) {
      const float3 rk = axpy3(-a, ld3(V.q, k), ld3(V.r[cur], k));
      st3(V.r[cur ^ 1], k, rk);
      st3(V.x, k, axpy3(a, ld3(V.p[pc ^ 1], k), ld3(V.x, k)));
      const float3 ru = cinv(A.C + (size_t)6 * k, rk);
      rrf += dot3(ru, ru);
      if (LPC) {
        st3(V.y, k, lower_row(G, A, V.r[cur], V.q, a, k, rk));
      } else {
        st3(V.z, k, rk);
        rzf += dot3(rk, rk);
      }
    }
    const float brr = block_sum<float, PN_THREADS>(rrf, sh);
    if (threadIdx.x == 0) prr[blockIdx.x] = brr;
    if (LPC) {
      ok = grid_barrier(P.bar, nblk, gen);
      if (!ok) break;
      // C: z = G^T y, r'.z
      for (int k = tid; k < K; k += nth) {
        const float3 z = upper_row(G, A, V.cu, V.y, k);
        st3(V.z, k, z);
        rzf += dot3(ld3(V.r[cur ^ 1], k), z);
      }
    }
    const float brz = block_sum<float, PN_THREADS>(rzf, sh);
    if (threadIdx.x == 0) prz[blockIdx.x] = brz;
    ok = grid_barrier(P.bar, nblk, gen);
    if (!ok) break;
    grid_sums<2, float, PN_THREADS>(fp, P32_MAXB, nblk, gs, sh);
    const float rz_new = gs[0];
    rr = gs[1];
    beta = rz != 0.f ? rz_new / rz : 0.f;
    rz = rz_new;
    cur ^= 1;
    pc ^= 1;
    ++it;
    done = rr <= tol2 * bb;
  }
  if (!ok) {
    if (tid == 0) set_status(status, ST_TIMEOUT);
    return;
  }
  for (int k = tid; k < K; k += nth) {
    const float3 x = ctmul(A.C + (size_t)6 * k, ld3(V.x, k));
    const double v[5] = {(double)x.x, (double)x.y, (double)x.z, 0.0, 0.0};
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      const size_t o = (size_t)r * K + k;
      P.x[o] = (float)v[r];  // as k_pcg32.cu leaves it (k_p32_finish reads it)
      out[o] = v[r];
      if (acc) acc[o] += v[r];
    }
  }
  __syncthreads();
  if (tid == 0) {
    P.scal[0] = rz;
    P.scal[3] = rr;
    P.scal[4] = bb;
    P.scal[5] = tol2;
    P.iter[0] = it;
    P.iter[1] = 1;
  }
}

int pcgn_blocks(bool lpc) {
  const void *f = lpc ? (const void *)k_pcgn<true> : (const void *)k_pcgn<false>;
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, f, PN_THREADS, 0) != cudaSuccess) return 0;
  return std::min(sms * per, P32_MAXB);
}

cudaError_t launch_pcgn(const LpcGraph &G, const LpcAct &A, const DevPCGN &V, const DevPCG32 &P, bool lpc,
                        const double *rhs, const double *x0, double rtol, int max_iters, double *out, double *acc,
                        int *status, int nblocks, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(P.bar, 0, 4 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  void *args[] = {(void *)&G, (void *)&A, (void *)&V, (void *)&P, (void *)&rhs, (void *)&x0, (void *)&rtol,
                  (void *)&max_iters, (void *)&out, (void *)&acc, (void *)&status};
  const void *f = lpc ? (const void *)k_pcgn<true> : (const void *)k_pcgn<false>;
  return cudaLaunchCooperativeKernel(f, dim3(nblocks), dim3(PN_THREADS), args, 0, s);
}

}  // namespace mabd
