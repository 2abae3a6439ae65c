// p2p.cu -- near field: direct 1/r interactions between a target leaf and
// the source leaves of its P2P list (Sec. II.A; Sec. II.C: P2P only needs
// the neighbours).
//
// One block of 128 threads per target leaf (targets in chunks of 256).  Each
// thread owns two targets (i and i + T2, T2 = ceil(n/2)), so one shared-memory
// load of a source serves two pairs.  The T2 threads of a target chunk form a
// group; G = floor(128 / T2) groups split every staged source tile into G
// contiguous pieces, and the G partial sums are added in a fixed order at the
// end (results are reproducible).  Sources are streamed through shared
// memory in tiles of 512 bodies (float4, 16-byte cp.async copies, double
// buffered): first the leaf's own bodies (masked: self and coincident pairs
// contribute zero), then the merged neighbour ranges back to back.  Bodies of
// two different leaves never coincide, so those tiles need no mask.
// Within a tile each thread sums naively; tile sums are combined with
// compensated (Kahan) addition.
#include "kernels.cuh"

namespace gbfmm {
namespace {

constexpr int kThreads = 128;
constexpr int kTgtChunk = 2 * kThreads;
constexpr int kSrcTile = 512;

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
__device__ __forceinline__ void pair(const R4& b, R xi, R yi, R zi, Acc<R>& a) {
  const R dx = b.x - xi, dy = b.y - yi, dz = b.z - zi;
  const R r2 = dx * dx + dy * dy + dz * dz;
  R inv = rsqrt_fast(r2);
  if (MASK) inv = r2 > (R)0 ? inv : (R)0;
  const R qi = b.w * inv;
  a.p += qi;
  const R f = qi * inv * inv;
  a.x += f * dx;
  a.y += f * dy;
  a.z += f * dz;
}

template <class R, class R4, bool MASK>
__device__ __forceinline__ void tile_sum(const R4* __restrict__ src, int k0, int k1, R xa, R ya, R za, R xb,
                                         R yb, R zb, Acc<R>& pa, Acc<R>& pb) {
#pragma unroll 4
  for (int k = k0; k < k1; ++k) {
    const R4 b = src[k];
    pair<R, R4, MASK>(b, xa, ya, za, pa);
    pair<R, R4, MASK>(b, xb, yb, zb, pb);
  }
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
template <class R4>
__device__ __forceinline__ void copy_body(R4* dst, const R4* src) {
  if (sizeof(R4) == 16) {
    cp_async16(dst, src);
  } else {
    cp_async16(dst, src);
    cp_async16(reinterpret_cast<char*>(dst) + 16, reinterpret_cast<const char*>(src) + 16);
  }
}

// Source stream of one leaf: the neighbour ranges [r0, r1) back to back.
struct Cursor {
  int r, off;
};

// Fill one tile from the stream; returns the number of bodies (uniform over
// the block: every thread walks the same ranges).
template <class R4>
__device__ __forceinline__ int fill_tile(R4* tile, const R4* __restrict__ bodies, const int2* __restrict__ ranges,
                                         Cursor& cur, int r1, const Lim& lim) {
  int filled = 0;
  while (filled < kSrcTile && cur.r < r1) {
    const int2 rg = GB_LD(ranges, cur.r, lim.nranges, 107);
    const int b = rg.x + cur.off;
    const int take = min(rg.y - b, kSrcTile - filled);
    for (int k = threadIdx.x; k < take; k += kThreads) {
#ifdef GBFMM_CHECKED
      if (!in_range(b + k, lim.N, 108, lim.rec)) continue;
#endif
      copy_body(tile + filled + k, bodies + b + k);
    }
    filled += take;
    if (b + take == rg.y) {
      ++cur.r;
      cur.off = 0;
    } else {
      cur.off += take;
    }
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  return filled;
}

template <class R, class R4>
__global__ void __launch_bounds__(kThreads) k_p2p(const R4* __restrict__ bodies, const int32_t* __restrict__ leaves,
                                                  const int32_t* __restrict__ bbeg, const int32_t* __restrict__ bend,
                                                  const int32_t* __restrict__ rptr, const int2* __restrict__ ranges,
                                                  R4* __restrict__ near, Lim lim) {
  __shared__ R4 tiles[2][kSrcTile];
  __shared__ Acc<R> red[2][kThreads];
  const int li = blockIdx.x;
  const int cell = GB_LD(leaves, li, lim.nleaf, 101);
  const int s = GB_LD(bbeg, cell, lim.ncell, 102), e = GB_LD(bend, cell, lim.ncell, 103);
  const int r0 = GB_LD(rptr, li, lim.nleaf + 1, 104), r1 = GB_LD(rptr, li + 1, lim.nleaf + 1, 105);
  const int tid = threadIdx.x;
  for (int t0 = s; t0 < e; t0 += kTgtChunk) {
    const int nt = min(kTgtChunk, e - t0);
    const int T2 = (nt + 1) >> 1;
    const int G = kThreads / T2;
    const int i = tid % T2, g = tid / T2;
    const bool active = g < G;
    const bool has_b = i + T2 < nt;
    R xa = 0, ya = 0, za = 0, xb = 0, yb = 0, zb = 0;
    if (active) {
      const R4 a = GB_LD(bodies, t0 + i, lim.N, 106);
      xa = a.x;
      ya = a.y;
      za = a.z;
      const R4 b = has_b ? GB_LD(bodies, t0 + i + T2, lim.N, 106) : a;
      xb = b.x;
      yb = b.y;
      zb = b.z;
    }
    Acc<R> sa{0, 0, 0, 0}, ca{0, 0, 0, 0}, sb{0, 0, 0, 0}, cb{0, 0, 0, 0};
    // own leaf, masked (tiles of the leaf's bodies)
    for (int c0 = s; c0 < e; c0 += kSrcTile) {
      const int cnt = min(kSrcTile, e - c0);
      __syncthreads();
      for (int k = tid; k < cnt; k += kThreads) copy_body(&tiles[0][k], bodies + c0 + k);
      asm volatile("cp.async.commit_group;\n" ::: "memory");
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
      __syncthreads();
      if (active) {
        const int k0 = (g * cnt) / G, k1 = ((g + 1) * cnt) / G;
        Acc<R> pa{0, 0, 0, 0}, pb{0, 0, 0, 0};
        tile_sum<R, R4, true>(tiles[0], k0, k1, xa, ya, za, xb, yb, zb, pa, pb);
        kahan_add(sa, ca, pa);
        kahan_add(sb, cb, pb);
      }
    }
    // neighbour stream, double buffered
    Cursor cur{r0, 0};
    __syncthreads();
    int cnt = fill_tile(tiles[0], bodies, ranges, cur, r1, lim);
    int buf = 0;
    while (cnt > 0) {
      const int nxt = fill_tile(tiles[buf ^ 1], bodies, ranges, cur, r1, lim);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
      __syncthreads();
      if (active) {
        const int k0 = (g * cnt) / G, k1 = ((g + 1) * cnt) / G;
        Acc<R> pa{0, 0, 0, 0}, pb{0, 0, 0, 0};
        tile_sum<R, R4, false>(tiles[buf], k0, k1, xa, ya, za, xb, yb, zb, pa, pb);
        kahan_add(sa, ca, pa);
        kahan_add(sb, cb, pb);
      }
      __syncthreads();  // tiles[buf] is refilled two steps later
      buf ^= 1;
      cnt = nxt;
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    red[0][tid] = sa;
    red[1][tid] = sb;
    __syncthreads();
    if (active && g == 0) {
      Acc<R> ta = red[0][i], tb = red[1][i];
      for (int gg = 1; gg < G; ++gg) {
        const Acc<R> va = red[0][gg * T2 + i], vb = red[1][gg * T2 + i];
        ta.p += va.p; ta.x += va.x; ta.y += va.y; ta.z += va.z;
        tb.p += vb.p; tb.x += vb.x; tb.y += vb.y; tb.z += vb.z;
      }
      R4 o;
      o.x = ta.p; o.y = ta.x; o.z = ta.y; o.w = ta.z;
      GB_ST(near, t0 + i, lim.N, 109, o);
      if (has_b) {
        o.x = tb.p; o.y = tb.x; o.z = tb.y; o.w = tb.z;
        GB_ST(near, t0 + i + T2, lim.N, 109, o);
      }
    }
    __syncthreads();
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
