// Grid-wide synchronisation of a cooperative launch (all blocks
// co-resident) with bounded waits, and deterministic sums over the grid.
#pragma once
#include "mabd_internal.h"

namespace mabd {

constexpr int P32_THREADS = 256;  // threads per block of the persistent solves

// Grid barrier over the co-resident blocks of a cooperative launch: bar[0]
// counts arrivals over the whole launch (zeroed before it), so barrier g is
// passed once it reaches (g + 1) * blocks; bar[2] is an error flag.  A wait
// gives up after P32_BAR_SPINS polls (about a second), sets the flag and
// returns false; every block then leaves the solve at its next barrier.
constexpr unsigned P32_BAR_SPINS = 1u << 22;

__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned nblk, unsigned &gen) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *vb = bar;
    const unsigned target = (gen + 1) * nblk;
    __threadfence();
    atomicAdd(&bar[0], 1u);
    unsigned spins = 0;
    while (vb[0] < target) {
      if (++spins > P32_BAR_SPINS) {
        atomicExch(&bar[2], 1u);
        break;
      }
    }
    __threadfence();
    ok_s = vb[2] == 0u;
  }
  __syncthreads();
  ++gen;
  return ok_s != 0;
}

// sums over the block of NV values per thread (every thread gets them):
// warp shuffles, then one pass over the warps' sums (T = float or double)
template <int NV, typename T, int NT = P32_THREADS>
__device__ __forceinline__ void block_sums(T (&v)[NV], T *sh) {
  constexpr int NW = NT / 32;
#pragma unroll
  for (int i = 0; i < NV; ++i)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) sh[i * NW + w] = v[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    T t = T(0);
#pragma unroll
    for (int q = 0; q < NW; ++q) t += sh[i * NW + q];
    v[i] = t;
  }
  __syncthreads();
}

template <typename T, int NT = P32_THREADS>
__device__ __forceinline__ T block_sum(T v, T *sh) {
  T a[1] = {v};
  block_sums<1, T, NT>(a, sh);
  return a[0];
}

// the grid's sums of NV sets of per-block partials part[i * stride + 0 .. n):
// every block adds them in the same order, so every block holds the same
// values
template <int NV, typename T, int NT = P32_THREADS>
__device__ __forceinline__ void grid_sums(const T *part, int stride, int n, T (&v)[NV], T *sh) {
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    v[i] = T(0);
    for (int b = threadIdx.x; b < n; b += NT) v[i] += ((const volatile T *)part)[i * stride + b];
  }
  block_sums<NV, T, NT>(v, sh);
}

template <typename T, int NT = P32_THREADS>
__device__ __forceinline__ T grid_sum(const T *part, int n, T *sh) {
  T a[1];
  grid_sums<1, T, NT>(part, 0, n, a, sh);
  return a[0];
}

}  // namespace mabd
