// p2p.cu -- near field: direct 1/r interactions between a target leaf and
// the source leaves of its P2P list (Sec. II.A; Sec. II.C: P2P only needs
// the neighbours).
//
// One block of 128 threads per target leaf.  A leaf of n <= 128 bodies is
// covered G = floor(128 / n) times: thread (g, i) accumulates target i over
// the sources j = g, g + G, ... of every staged tile, and the G partial sums
// are added in a fixed order at the end (so results are reproducible).
// Sources are staged through shared memory in tiles of 256 bodies (16 B
// float4 each, coalesced loads).  Within a tile each thread sums naively; the
// tile sums are combined with compensated (Kahan) addition.  The leaf's own
// bodies are a separate, masked pass (self and coincident pairs contribute
// zero); bodies of two different leaves always differ in position, so the
// other ranges need no mask.
#include "kernels.cuh"

namespace gbfmm {
namespace {

constexpr int kThreads = 128;
constexpr int kSrcTile = 256;

__device__ __forceinline__ float rsqrt_fast(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double rsqrt_fast(double x) { return rsqrt(x); }

template <class R>
struct Acc {
  R p, x, y, z;
};

template <class R>
__device__ __forceinline__ void kahan_add(Acc<R>& s, Acc<R>& c, const Acc<R>& v) {
  R y, t;
  y = v.p - c.p; t = s.p + y; c.p = (t - s.p) - y; s.p = t;
  y = v.x - c.x; t = s.x + y; c.x = (t - s.x) - y; s.x = t;
  y = v.y - c.y; t = s.y + y; c.y = (t - s.y) - y; s.y = t;
  y = v.z - c.z; t = s.z + y; c.z = (t - s.z) - y; s.z = t;
}

template <class R, class R4, bool MASK>
__device__ __forceinline__ void tile_sum(const R4* __restrict__ src, int cnt, int g, int G, R xi, R yi, R zi,
                                         Acc<R>& part) {
#pragma unroll 4
  for (int k = g; k < cnt; k += G) {
    const R4 b = src[k];
    const R dx = b.x - xi, dy = b.y - yi, dz = b.z - zi;
    const R r2 = dx * dx + dy * dy + dz * dz;
    R inv = rsqrt_fast(r2);
    if (MASK) inv = r2 > (R)0 ? inv : (R)0;
    const R qi = b.w * inv;
    part.p += qi;
    const R f = qi * inv * inv;
    part.x += f * dx;
    part.y += f * dy;
    part.z += f * dz;
  }
}

template <class R, class R4>
__global__ void __launch_bounds__(kThreads) k_p2p(const R4* __restrict__ bodies, const int32_t* __restrict__ leaves,
                                                  const int32_t* __restrict__ bbeg, const int32_t* __restrict__ bend,
                                                  const int32_t* __restrict__ rptr, const int2* __restrict__ ranges,
                                                  R4* __restrict__ near, Lim lim) {
  __shared__ R4 src[kSrcTile];
  __shared__ Acc<R> red[kThreads];
  const int li = blockIdx.x;
  const int cell = GB_LD(leaves, li, lim.nleaf, 101);
  const int s = GB_LD(bbeg, cell, lim.ncell, 102), e = GB_LD(bend, cell, lim.ncell, 103);
  const int r0 = GB_LD(rptr, li, lim.nleaf + 1, 104), r1 = GB_LD(rptr, li + 1, lim.nleaf + 1, 105);
  const int tid = threadIdx.x;
  for (int t0 = s; t0 < e; t0 += kThreads) {
    const int nt = min(kThreads, e - t0);
    const int G = kThreads / nt;
    const int ti = tid % nt, g = tid / nt;
    const bool active = g < G;
    R xi = 0, yi = 0, zi = 0;
    if (active) {
      const R4 b = GB_LD(bodies, t0 + ti, lim.N, 106);
      xi = b.x;
      yi = b.y;
      zi = b.z;
    }
    Acc<R> sum{0, 0, 0, 0}, cmp{0, 0, 0, 0};
    // own leaf (masked), then the merged neighbour ranges
    for (int r = r0 - 1; r < r1; ++r) {
      int b0, b1;
      if (r < r0) {
        b0 = s;
        b1 = e;
      } else {
        const int2 rg = GB_LD(ranges, r, lim.nranges, 107);
        b0 = rg.x;
        b1 = rg.y;
      }
      for (int c0 = b0; c0 < b1; c0 += kSrcTile) {
        const int cnt = min(kSrcTile, b1 - c0);
        __syncthreads();
        for (int k = tid; k < cnt; k += kThreads) src[k] = GB_LD(bodies, c0 + k, lim.N, 108);
        __syncthreads();
        if (active) {
          Acc<R> part{0, 0, 0, 0};
          if (r < r0) tile_sum<R, R4, true>(src, cnt, g, G, xi, yi, zi, part);
          else tile_sum<R, R4, false>(src, cnt, g, G, xi, yi, zi, part);
          kahan_add(sum, cmp, part);
        }
      }
    }
    __syncthreads();
    red[tid] = sum;
    __syncthreads();
    if (active && g == 0) {
      Acc<R> tot = red[ti];
      for (int gg = 1; gg < G; ++gg) {
        const Acc<R> v = red[gg * nt + ti];
        tot.p += v.p;
        tot.x += v.x;
        tot.y += v.y;
        tot.z += v.z;
      }
      R4 o;
      o.x = tot.p;
      o.y = tot.x;
      o.z = tot.y;
      o.w = tot.z;
      GB_ST(near, t0 + ti, lim.N, 109, o);
    }
  }
}

}  // namespace

template <class R>
void launch_p2p(fmm_tree* t, cudaStream_t s) {
  using R4 = typename Vec4<R>::type;
  k_p2p<R, R4><<<t->nleaf, kThreads, 0, s>>>((const R4*)t->work, t->leaves, t->c.bbeg, t->c.bend, t->p2p_rptr,
                                             t->p2p_ranges, (R4*)t->near, t->lim);
  GB_LAUNCH("k_p2p");
}

template void launch_p2p<float>(fmm_tree*, cudaStream_t);
template void launch_p2p<double>(fmm_tree*, cudaStream_t);

}  // namespace gbfmm
