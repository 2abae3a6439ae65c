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

// ---------------------------------------------------------------------------
// Single precision with packed FP32 pairs (add/sub/mul/fma.rn.f32x2, sm_100
// and later): one instruction evaluates one target against two sources.  The
// staged tile holds the sources two by two, {x0,x1,y0,y1} {z0,z1,q0,q1}, so a
// pair of sources is two 16-byte shared loads.  Each thread owns two targets
// as in the generic kernel; its sums are kept per source parity (the low and
// high halves) and added at the end.  A padding source (odd tile length) sits
// at 1e30 with zero charge: r^2 overflows to +inf, rsqrt gives 0, and it adds
// exactly zero.

typedef unsigned long long f2;  // two packed floats (low half first in memory)

__device__ __forceinline__ f2 f2_pack(float lo, float hi) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(f2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  f2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
  f2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  f2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
  f2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

struct Acc2 {
  f2 p, x, y, z;
};

// One target (X, Y, Z duplicated in both halves) against the source pair.
template <bool MASK>
__device__ __forceinline__ void pair2(f2 XX, f2 YY, f2 ZZ, f2 QQ, f2 X, f2 Y, f2 Z, Acc2& a) {
  const f2 dx = f2_sub(XX, X), dy = f2_sub(YY, Y), dz = f2_sub(ZZ, Z);
  f2 r2 = f2_mul(dx, dx);
  r2 = f2_fma(dy, dy, r2);
  r2 = f2_fma(dz, dz, r2);
  float rl, rh;
  f2_unpack(r2, rl, rh);
  float il = rsqrt_fast(rl), ih = rsqrt_fast(rh);
  if (MASK) {
    il = rl > 0.f ? il : 0.f;
    ih = rh > 0.f ? ih : 0.f;
  }
  const f2 inv = f2_pack(il, ih);
  const f2 qi = f2_mul(QQ, inv);
  a.p = f2_add(a.p, qi);
  const f2 f = f2_mul(f2_mul(qi, inv), inv);
  a.x = f2_fma(f, dx, a.x);
  a.y = f2_fma(f, dy, a.y);
  a.z = f2_fma(f, dz, a.z);
}

constexpr int kPairTile = kSrcTile / 2;
constexpr int kSlots = kSrcTile / kThreads;  // bodies staged per thread per tile
constexpr float kFar = 1e30f;

struct __align__(16) SrcPair {
  float w[8];  // x0 x1 y0 y1 z0 z1 q0 q1
};

__device__ __forceinline__ void put_body(SrcPair* tile, int slot, float4 b) {
  float* w = tile[slot >> 1].w + (slot & 1);
  w[0] = b.x;
  w[2] = b.y;
  w[4] = b.z;
  w[6] = b.w;
}

// Global indices of this thread's slots of the next tile of the neighbour
// stream (-1: none); returns the tile length (uniform over the block).
__device__ __forceinline__ int plan_tile(const int2* __restrict__ ranges, Cursor& cur, int r1, int (&gidx)[kSlots],
                                         const Lim& lim) {
  int filled = 0;
#pragma unroll
  for (int m = 0; m < kSlots; ++m) gidx[m] = -1;
  while (filled < kSrcTile && cur.r < r1) {
    const int2 rg = GB_LD(ranges, cur.r, lim.nranges, 107);
    const int b = rg.x + cur.off;
    const int take = min(rg.y - b, kSrcTile - filled);
#pragma unroll
    for (int m = 0; m < kSlots; ++m) {
      const int sl = threadIdx.x + m * kThreads - filled;
      if (sl >= 0 && sl < take) gidx[m] = b + sl;
    }
    filled += take;
    if (b + take == rg.y) {
      ++cur.r;
      cur.off = 0;
    } else {
      cur.off += take;
    }
  }
  return filled;
}

// The same plan from the leaf's ranges staged in shared memory with their
// exclusive prefix sums (pre[r] = bodies before range r): stream position S
// lies in the last range r with pre[r] <= S.  Each thread's positions only
// grow (slots within a tile, then tiles), so its cursor r only moves
// forward: planning costs O(ranges + slots) per leaf and thread instead of
// a walk over every range for every tile.
constexpr int kStagedRanges = 256;

__device__ __forceinline__ int plan_tile_staged(const int2* __restrict__ rng, const int* __restrict__ pre, int nr,
                                                int T, int& cur, int (&gidx)[kSlots]) {
  const int total = pre[nr];
  const int cnt = min(kSrcTile, total - T);
#pragma unroll
  for (int m = 0; m < kSlots; ++m) {
    const int sl = threadIdx.x + m * kThreads;
    gidx[m] = -1;
    if (sl < cnt) {
      const int S = T + sl;
      while (pre[cur + 1] <= S) ++cur;
      gidx[m] = rng[cur].x + (S - pre[cur]);
    }
  }
  return cnt > 0 ? cnt : 0;
}

__device__ __forceinline__ void load_slots(const float4* __restrict__ bodies, const int (&gidx)[kSlots],
                                           float4 (&v)[kSlots], const Lim& lim) {
#pragma unroll
  for (int m = 0; m < kSlots; ++m)
    v[m] = gidx[m] >= 0 ? GB_LD(bodies, gidx[m], lim.N, 108) : make_float4(kFar, kFar, kFar, 0.f);
}

__device__ __forceinline__ void store_slots(SrcPair* tile, int cnt, const float4 (&v)[kSlots]) {
  const int lim2 = (cnt + 1) & ~1;  // slots up to the even length (the pad)
#pragma unroll
  for (int m = 0; m < kSlots; ++m) {
    const int sl = threadIdx.x + m * kThreads;
    if (sl < lim2) put_body(tile, sl, v[m]);
  }
}

template <bool MASK>
__device__ __forceinline__ void tile_sum2(const SrcPair* __restrict__ tile, int k0, int k1, f2 X0, f2 Y0, f2 Z0,
                                          f2 X1, f2 Y1, f2 Z1, Acc2& a0, Acc2& a1) {
#pragma unroll 2
  for (int k = k0; k < k1; ++k) {
    const ulonglong2 A = *reinterpret_cast<const ulonglong2*>(tile[k].w);
    const ulonglong2 B = *reinterpret_cast<const ulonglong2*>(tile[k].w + 4);
    pair2<MASK>(A.x, A.y, B.x, B.y, X0, Y0, Z0, a0);
    pair2<MASK>(A.x, A.y, B.x, B.y, X1, Y1, Z1, a1);
  }
}

__global__ void __launch_bounds__(kThreads) k_p2p_f2(const float4* __restrict__ bodies,
                                                     const int32_t* __restrict__ leaves,
                                                     const int32_t* __restrict__ bbeg, const int32_t* __restrict__ bend,
                                                     const int32_t* __restrict__ rptr, const int2* __restrict__ ranges,
                                                     float4* __restrict__ near, Lim lim) {
  __shared__ SrcPair tiles[2][kPairTile];
  __shared__ Acc<float> red[2][kThreads];
  __shared__ int2 srng[kStagedRanges];
  __shared__ int spre[kStagedRanges + 1];
  const int li = blockIdx.x;
  const int cell = GB_LD(leaves, li, lim.nleaf, 101);
  const int s = GB_LD(bbeg, cell, lim.ncell, 102), e = GB_LD(bend, cell, lim.ncell, 103);
  const int r0 = GB_LD(rptr, li, lim.nleaf + 1, 104), r1 = GB_LD(rptr, li + 1, lim.nleaf + 1, 105);
  const int tid = threadIdx.x;
  const f2 zero = 0ull;
  // the leaf's neighbour ranges and their prefix sums in shared memory (warp
  // 0 scans 32 ranges at a time); larger lists take the uniform range walk
  const int nr = r1 - r0;
  const bool staged = nr <= kStagedRanges;
  if (staged && tid < 32) {
    int base = 0;
    for (int r = tid; r - tid < nr; r += 32) {
      int len = 0;
      if (r < nr) {
        const int2 rg = GB_LD(ranges, r0 + r, lim.nranges, 107);
        srng[r] = rg;
        len = rg.y - rg.x;
      }
      int incl = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (tid >= o) incl += v;
      }
      if (r < nr) spre[r] = base + incl - len;
      base += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (tid == 0) spre[nr] = base;
  }
  __syncthreads();
  for (int t0 = s; t0 < e; t0 += kTgtChunk) {
    const int nt = min(kTgtChunk, e - t0);
    const int T2 = (nt + 1) >> 1;
    const int G = kThreads / T2;
    const int i = tid % T2, g = tid / T2;
    const bool active = g < G;
    const bool has_b = i + T2 < nt;
    f2 X0 = zero, Y0 = zero, Z0 = zero, X1 = zero, Y1 = zero, Z1 = zero;
    if (active) {
      const float4 a = GB_LD(bodies, t0 + i, lim.N, 106);
      const float4 b = has_b ? GB_LD(bodies, t0 + i + T2, lim.N, 106) : a;
      X0 = f2_pack(a.x, a.x);
      Y0 = f2_pack(a.y, a.y);
      Z0 = f2_pack(a.z, a.z);
      X1 = f2_pack(b.x, b.x);
      Y1 = f2_pack(b.y, b.y);
      Z1 = f2_pack(b.z, b.z);
    }
    // tile sums: the two parities folded, then compensated (Kahan) addition
    auto fold = [](const Acc2& a) {
      Acc<float> r;
      float l, h;
      f2_unpack(a.p, l, h);
      r.p = l + h;
      f2_unpack(a.x, l, h);
      r.x = l + h;
      f2_unpack(a.y, l, h);
      r.y = l + h;
      f2_unpack(a.z, l, h);
      r.z = l + h;
      return r;
    };
    Acc<float> s0{0, 0, 0, 0}, c0{0, 0, 0, 0}, s1{0, 0, 0, 0}, c1{0, 0, 0, 0};
    auto accumulate = [&](const Acc2& p, Acc<float>& sm, Acc<float>& cm) { kahan_add(sm, cm, fold(p)); };
    // own leaf, masked
    for (int c0b = s; c0b < e; c0b += kSrcTile) {
      const int cnt = min(kSrcTile, e - c0b);
      int gidx[kSlots];
#pragma unroll
      for (int m = 0; m < kSlots; ++m) {
        const int sl = tid + m * kThreads;
        gidx[m] = sl < cnt ? c0b + sl : -1;
      }
      float4 v[kSlots];
      load_slots(bodies, gidx, v, lim);
      __syncthreads();
      store_slots(tiles[0], cnt, v);
      __syncthreads();
      if (active) {
        const int np = (cnt + 1) >> 1;
        const int k0 = (g * np) / G, k1 = ((g + 1) * np) / G;
        Acc2 p0{zero, zero, zero, zero}, p1{zero, zero, zero, zero};
        tile_sum2<true>(tiles[0], k0, k1, X0, Y0, Z0, X1, Y1, Z1, p0, p1);
        accumulate(p0, s0, c0);
        accumulate(p1, s1, c1);
      }
    }
    // neighbour stream: the next tile is loaded into registers while the
    // current one is summed
    Cursor cur{r0, 0};
    int scur = 0, T = 0;
    auto plan = [&](int (&gi)[kSlots]) {
      if (staged) {
        const int c = plan_tile_staged(srng, spre, nr, T, scur, gi);
        T += kSrcTile;
        return c;
      }
      return plan_tile(ranges, cur, r1, gi, lim);
    };
    int gidx[kSlots];
    float4 v[kSlots];
    int cnt = plan(gidx);
    load_slots(bodies, gidx, v, lim);
    __syncthreads();
    store_slots(tiles[0], cnt, v);
    __syncthreads();
    int buf = 0;
    while (cnt > 0) {
      const int nxt = plan(gidx);
      if (nxt > 0) load_slots(bodies, gidx, v, lim);
      if (active) {
        const int np = (cnt + 1) >> 1;
        const int k0 = (g * np) / G, k1 = ((g + 1) * np) / G;
        Acc2 p0{zero, zero, zero, zero}, p1{zero, zero, zero, zero};
        tile_sum2<false>(tiles[buf], k0, k1, X0, Y0, Z0, X1, Y1, Z1, p0, p1);
        accumulate(p0, s0, c0);
        accumulate(p1, s1, c1);
      }
      // tiles[buf ^ 1] was last read two iterations ago (before the barrier
      // that ended the previous iteration)
      if (nxt > 0) store_slots(tiles[buf ^ 1], nxt, v);
      __syncthreads();
      buf ^= 1;
      cnt = nxt;
    }
    red[0][tid] = s0;
    red[1][tid] = s1;
    __syncthreads();
    if (active && g == 0) {
      Acc<float> ta = red[0][i], tb = red[1][i];
      for (int gg = 1; gg < G; ++gg) {
        const Acc<float> va = red[0][gg * T2 + i], vb = red[1][gg * T2 + i];
        ta.p += va.p; ta.x += va.x; ta.y += va.y; ta.z += va.z;
        tb.p += vb.p; tb.x += vb.x; tb.y += vb.y; tb.z += vb.z;
      }
      GB_ST(near, t0 + i, lim.N, 109, make_float4(ta.p, ta.x, ta.y, ta.z));
      if (has_b) GB_ST(near, t0 + i + T2, lim.N, 109, make_float4(tb.p, tb.x, tb.y, tb.z));
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Mutual interaction (FMM_FLAG_MUTUAL_P2P): a block per unordered leaf pair
// (A, B), A < B, computes each body pair once and updates both sides: the
// target side in registers (thread per body of A), the source side in
// shared memory, where thread i at step k takes body (i + k) mod n of the
// staged tile of B so that a warp's updates hit distinct addresses.  Every
// result reaches `near` through atomic additions (near starts at zero), so
// the order of the additions, and the last bits, vary from run to run.
// Blocks past the pairs take one leaf each: its self interaction, one-sided
// and masked.
template <class R>
__device__ __forceinline__ void atomic_add4(typename Vec4<R>::type* p, R a, R b, R c, R d) {
  R* q = reinterpret_cast<R*>(p);
  atomicAdd(q + 0, a);
  atomicAdd(q + 1, b);
  atomicAdd(q + 2, c);
  atomicAdd(q + 3, d);
}

template <class R, class R4>
__global__ void __launch_bounds__(kThreads) k_p2p_mutual(const R4* __restrict__ bodies,
                                                         const int2* __restrict__ upairs, int64_t nup,
                                                         const int32_t* __restrict__ leaves,
                                                         const int32_t* __restrict__ bbeg,
                                                         const int32_t* __restrict__ bend, R4* __restrict__ near,
                                                         Lim lim) {
  __shared__ R4 tile[kSrcTile];
  __shared__ R acc[4][kSrcTile];
  const int tid = threadIdx.x;
  const int64_t b = blockIdx.x;
  if (b >= nup) {
    // self interaction of one leaf
    const int cell = GB_LD(leaves, (int)(b - nup), lim.nleaf, 111);
    const int s = GB_LD(bbeg, cell, lim.ncell, 112), e = GB_LD(bend, cell, lim.ncell, 113);
    for (int t0 = s; t0 < e; t0 += kThreads) {
      const int i = t0 + tid;
      Acc<R> a{0, 0, 0, 0};
      const bool act = i < e;
      const R4 bi = act ? GB_LD(bodies, i, lim.N, 114) : R4{};
      for (int c0 = s; c0 < e; c0 += kSrcTile) {
        const int cnt = min(kSrcTile, e - c0);
        __syncthreads();
        for (int k = tid; k < cnt; k += kThreads) tile[k] = GB_LD(bodies, c0 + k, lim.N, 115);
        __syncthreads();
        if (act)
          for (int k = 0; k < cnt; ++k) pair<R, R4, true>(tile[k], bi.x, bi.y, bi.z, a);
      }
      if (act) atomic_add4<R>(near + i, a.p, a.x, a.y, a.z);
    }
    return;
  }
  const int2 up = GB_LD(upairs, b, nup, 116);
  const int sA = GB_LD(bbeg, up.x, lim.ncell, 117), eA = GB_LD(bend, up.x, lim.ncell, 118);
  const int sB = GB_LD(bbeg, up.y, lim.ncell, 119), eB = GB_LD(bend, up.y, lim.ncell, 120);
  for (int b0 = sB; b0 < eB; b0 += kSrcTile) {
    const int nb = min(kSrcTile, eB - b0);
    __syncthreads();
    for (int k = tid; k < nb; k += kThreads) {
      tile[k] = GB_LD(bodies, b0 + k, lim.N, 121);
      acc[0][k] = acc[1][k] = acc[2][k] = acc[3][k] = (R)0;
    }
    __syncthreads();
    for (int a0 = sA; a0 < eA; a0 += kThreads) {
      const int i = a0 + tid;
      if (i < eA) {
        const R4 bi = GB_LD(bodies, i, lim.N, 122);
        R p = 0, ax = 0, ay = 0, az = 0;
        int j = tid % nb;
        for (int k = 0; k < nb; ++k) {
          const R4 bj = tile[j];
          const R dx = bj.x - bi.x, dy = bj.y - bi.y, dz = bj.z - bi.z;
          const R r2 = dx * dx + dy * dy + dz * dz;
          const R inv = rsqrt_fast(r2);  // bodies of two leaves never coincide
          const R inv3 = inv * inv * inv;
          p += bj.w * inv;
          const R fj = bj.w * inv3;
          ax += fj * dx;
          ay += fj * dy;
          az += fj * dz;
          // reaction on body j: potential q_i / r, gradient q_i (x_i - x_j) / r^3
          const R fi = bi.w * inv3;
          atomicAdd(&acc[0][j], bi.w * inv);
          atomicAdd(&acc[1][j], -fi * dx);
          atomicAdd(&acc[2][j], -fi * dy);
          atomicAdd(&acc[3][j], -fi * dz);
          j = j + 1 == nb ? 0 : j + 1;
        }
        atomic_add4<R>(near + i, p, ax, ay, az);
      }
    }
    __syncthreads();
    for (int k = tid; k < nb; k += kThreads) atomic_add4<R>(near + b0 + k, acc[0][k], acc[1][k], acc[2][k], acc[3][k]);
  }
}

}  // namespace

template <class R>
void launch_p2p(fmm_tree* t, cudaStream_t s) {
  using R4 = typename Vec4<R>::type;
  if (t->flags & FMM_FLAG_MUTUAL_P2P) {
    GB_CK(cudaMemsetAsync(t->near, 0, sizeof(R4) * (size_t)t->N, s));
    const int64_t nblk = t->n_p2p_upairs + t->nleaf;
    k_p2p_mutual<R, R4><<<(unsigned)nblk, kThreads, 0, s>>>((const R4*)t->work, t->p2p_upairs, t->n_p2p_upairs,
                                                            t->leaves, t->c.bbeg, t->c.bend, (R4*)t->near, t->lim);
    GB_LAUNCH("k_p2p_mutual");
    return;
  }
  if (std::is_same<R, float>::value) {
    k_p2p_f2<<<t->nleaf, kThreads, 0, s>>>((const float4*)t->work, t->leaves, t->c.bbeg, t->c.bend, t->p2p_rptr,
                                           t->p2p_ranges, (float4*)t->near, t->lim);
    GB_LAUNCH("k_p2p_f2");
    return;
  }
  k_p2p<R, R4><<<t->nleaf, kThreads, 0, s>>>((const R4*)t->work, t->leaves, t->c.bbeg, t->c.bend, t->p2p_rptr,
                                             t->p2p_ranges, (R4*)t->near, t->lim);
  GB_LAUNCH("k_p2p");
}

template void launch_p2p<float>(fmm_tree*, cudaStream_t);
template void launch_p2p<double>(fmm_tree*, cudaStream_t);

}  // namespace gbfmm
