// grid.cuh -- device helpers of the cooperative build kernels: a grid-wide
// barrier with a bounded wait, and block sums of per-block partial counts.
#pragma once

#include "common.cuh"

namespace gbfmm {

struct GridBar {
  unsigned count, gen, abort;  // zeroed before the launch
};

constexpr long long kGridWaitNs = 2000000000ll;  // 2 s: far beyond any real wait

__device__ __forceinline__ long long grid_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Barrier over all blocks of a cooperative launch (all of them resident).
// Thread 0 of the last block to arrive resets the count and advances the
// generation; the others wait for the generation to change, at most
// kGridWaitNs, or until another block has given up.  A wait that runs out
// sets kErrGrid in *err and the abort flag; the result is then false in
// every block that sees it, and the kernel must return.
__device__ __forceinline__ bool grid_barrier(GridBar* bar, int* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* gen = &bar->gen;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(&bar->count, 1u) == gridDim.x - 1) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      const long long t0 = grid_ns();
      while (*gen == g) {
        if (*(volatile unsigned*)&bar->abort || grid_ns() - t0 > kGridWaitNs) {
          atomicOr(err, kErrGrid);
          atomicExch(&bar->abort, 1u);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// For NV counts per block stored value-major (partial[v * n + block]): the
// sums over the blocks before `upto` and over all n blocks, in every thread.
// The partials were written by other blocks before a grid barrier, so they
// are read through L2.
template <class T, int NV>
__device__ void block_prefix_totals(const T* partial, int upto, int n, T before[NV], T total[NV]) {
  __shared__ T sb[NV][32], st[NV][32];
  T b[NV], t[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) b[v] = t[v] = 0;
  for (int j = threadIdx.x; j < n; j += blockDim.x)
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const T x = __ldcg(partial + (int64_t)v * n + j);
      t[v] += x;
      if (j < upto) b[v] += x;
    }
#pragma unroll
  for (int v = 0; v < NV; ++v)
    for (int o = 16; o > 0; o >>= 1) {
      b[v] += __shfl_down_sync(0xffffffffu, b[v], o);
      t[v] += __shfl_down_sync(0xffffffffu, t[v], o);
    }
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      sb[v][threadIdx.x >> 5] = b[v];
      st[v][threadIdx.x >> 5] = t[v];
    }
  __syncthreads();
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    before[v] = total[v] = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      before[v] += sb[v][w];
      total[v] += st[v][w];
    }
  }
  __syncthreads();
}

}  // namespace gbfmm
