// p2p.cu -- near field: direct 1/r interactions between a target leaf and
// the source leaves of its P2P list (Sec. II.A; Sec. II.C: P2P only needs
// the neighbours).
//
// Double precision (k_p2p): one block of 128 threads per target leaf
// (targets in chunks of 256).  Each thread owns two targets (i and i + T2,
// T2 = ceil(n/2)), so one shared-memory load of a source serves two pairs.
// The T2 threads of a target chunk form a group; G = floor(128 / T2) groups
// split every staged source tile into G contiguous pieces, and the G partial
// sums are added in a fixed order at the end (results are reproducible).
// Sources are streamed through shared memory in tiles of 512 bodies (16-byte
// cp.async copies, double buffered): first the leaf's own bodies (masked:
// self and coincident pairs contribute zero), then the merged neighbour
// ranges back to back.  Bodies of two different leaves never coincide, so
// those tiles need no mask.  Within a tile each thread sums naively; tile
// sums are combined with compensated (Kahan) addition.
//
// Single precision (k_p2p_f2, below): the same per-thread scheme on packed
// FP32 pairs, one block per work item (a chunk of at most 256 targets of one
// leaf, largest items first), with bulk-copied source tiles.
#include <algorithm>
#include <cstdlib>

#include "kernels.cuh"
#include "mbarrier.cuh"

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
// Single precision with packed FP32 pairs (the float2 add/mul/fma of sm_100
// and later, __fadd2_rn and friends): one instruction evaluates one target
// against two sources.  Sources are read from a pair-major copy of the sorted bodies (k_pair_bodies:
// pair m = bodies 2m and 2m + 1 as {x0,x1,y0,y1} {z0,z1,q0,q1}, 32 bytes), so a
// pair of sources is two 16-byte shared loads and a body range of the
// neighbour stream is a contiguous run of pairs.  Each run is copied to
// shared memory by one bulk copy (cp.async.bulk) per tile it touches, and the
// copies of a tile complete on the tile's mbarrier; while a tile is summed the
// next one is in flight (two buffers, one block barrier per tile).  A range
// with an odd first body (or an odd end) brings one body too many into its
// first (last) pair; once the tile has landed, that half is overwritten with a
// far-away zero charge.  Each thread owns two targets as in the generic
// kernel, and the G groups of a target chunk take the pairs of a tile
// round-robin.  Its sums are kept per source parity (the low and high halves)
// and folded at the end of each tile.

typedef float2 f2;  // two packed floats (.x: the low half)

__device__ __forceinline__ f2 f2_pack(float lo, float hi) { return make_float2(lo, hi); }
__device__ __forceinline__ void f2_unpack(f2 v, float& lo, float& hi) {
  lo = v.x;
  hi = v.y;
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }

struct Acc2 {
  f2 p, x, y, z;
};

// One target (its negated coordinates duplicated in both halves) against the
// source pair.
template <bool MASK>
__device__ __forceinline__ void pair2(f2 XX, f2 YY, f2 ZZ, f2 QQ, f2 NX, f2 NY, f2 NZ, Acc2& a) {
  const f2 dx = f2_add(XX, NX), dy = f2_add(YY, NY), dz = f2_add(ZZ, NZ);
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

constexpr int kTilePairs = 448;  // source pairs per staged tile (896 bodies, 14 KB; 7 blocks per SM)
constexpr int kWindow = 256;     // neighbour ranges staged at a time
constexpr float kFar = 1e30f;

struct __align__(16) SrcPair {
  float w[8];  // x0 x1 y0 y1 z0 z1 q0 q1
};

// The sorted bodies in pair-major form: pair m holds bodies 2m and 2m + 1
// (the high half of the last pair of an odd count is a far-away zero charge).
__global__ void k_pair_bodies(const float4* __restrict__ b, long long n, SrcPair* __restrict__ out) {
  const long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (2 * m >= n) return;
  const float4 u = b[2 * m];
  const float4 v = 2 * m + 1 < n ? b[2 * m + 1] : make_float4(kFar, kFar, kFar, 0.f);
  float4* o = reinterpret_cast<float4*>(out + m);
  o[0] = make_float4(u.x, v.x, u.y, v.y);
  o[1] = make_float4(u.z, v.z, u.w, v.w);
}

// A source stream in shared memory: body ranges [a, b) as pair ranges
// [a/2, (b+1)/2), each as (first pair, pad bits) -- bit 0: the low half of the
// first pair (body a - 1) is not in the range, bit 1: the high half of the
// last pair (body b) is not -- and the exclusive prefix sums of the pair
// counts (pre[n] = the stream length in pairs).
struct Stream {
  int2 rng[kWindow];
  int pre[kWindow + 1];
};

// Warp 0 stages ranges [r0, r0 + nw) of the list (nw <= kWindow); every lane
// returns the stream length.
__device__ __forceinline__ int stage_window(Stream& st, const int2* __restrict__ ranges, int r0, int nw,
                                            const Lim& lim) {
  const int lane = threadIdx.x;
  int base = 0;
  for (int r = lane; r - lane < nw; r += 32) {
    int len = 0;
    if (r < nw) {
      const int2 rg = GB_LD(ranges, r0 + r, lim.nranges, 107);
      const int ps = rg.x >> 1, pe = (rg.y + 1) >> 1;
      st.rng[r] = make_int2(ps, (rg.x & 1) | ((rg.y & 1) << 1));
      len = pe - ps;
    }
    int incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (r < nw) st.pre[r] = base + incl - len;
    base += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) st.pre[nw] = base;
  return base;
}

// Bulk copies of stream pairs [T0, T1) into a tile, one per range piece,
// completing on bar (whose expected bytes are set by the caller).
__device__ __forceinline__ void issue_tile(const Stream& st, int nw, int T0, int T1,
                                           const SrcPair* __restrict__ src, uint32_t dst, uint32_t bar,
                                           const Lim& lim) {
  for (int r = threadIdx.x; r < nw; r += kThreads) {
    const int pr = st.pre[r];
    const int a = max(pr, T0), b = min(st.pre[r + 1], T1);
    if (a < b) {
      const int first = st.rng[r].x + (a - pr);
#ifdef GBFMM_CHECKED
      if (!in_range(first + (b - a) - 1, (lim.N + 1) / 2, 108, lim.rec)) continue;
#endif
      bulk_g2s(dst + (uint32_t)(a - T0) * (uint32_t)sizeof(SrcPair), src + first,
               (uint32_t)(b - a) * (uint32_t)sizeof(SrcPair), bar);
    }
  }
}

// After the copies of pairs [T0, T1) have landed: a half that lies outside
// its range becomes a far-away zero charge (r^2 overflows to +inf, rsqrt
// gives 0, and the half adds exactly zero, masked or not).
__device__ __forceinline__ void pad_tile(const Stream& st, int nw, int T0, int T1, SrcPair* tile) {
  for (int r = threadIdx.x; r < nw; r += kThreads) {
    const int f = st.rng[r].y;
    if (f == 0) continue;
    const int a = st.pre[r], b = st.pre[r + 1] - 1;
    if ((f & 1) && a >= T0 && a < T1) {
      tile[a - T0].w[0] = kFar;
      tile[a - T0].w[6] = 0.f;
    }
    if ((f & 2) && b >= T0 && b < T1) {
      tile[b - T0].w[1] = kFar;
      tile[b - T0].w[7] = 0.f;
    }
  }
}

// Group g of G takes pairs g, g + G, g + 2G, ... of a tile of np pairs.
template <bool MASK>
__device__ __forceinline__ void tile_sum2(const SrcPair* __restrict__ tile, int k, int np, int G, f2 X0, f2 Y0,
                                          f2 Z0, f2 X1, f2 Y1, f2 Z1, Acc2& a0, Acc2& a1) {
#pragma unroll 4
  for (; k < np; k += G) {
    const float4 A = *reinterpret_cast<const float4*>(tile[k].w);
    const float4 B = *reinterpret_cast<const float4*>(tile[k].w + 4);
    const f2 XX = make_float2(A.x, A.y), YY = make_float2(A.z, A.w);
    const f2 ZZ = make_float2(B.x, B.y), QQ = make_float2(B.z, B.w);
    pair2<MASK>(XX, YY, ZZ, QQ, X0, Y0, Z0, a0);
    pair2<MASK>(XX, YY, ZZ, QQ, X1, Y1, Z1, a1);
  }
}

// Shared memory of one block of the per-block kernel.
struct BlockSmem {
  SrcPair tiles[2][kTilePairs];
  Stream st;
  unsigned long long bar[2];
  int abort_flag;
};

// One work item per block (the block-wide body of k_p2p_mix).
__device__ __forceinline__ void p2p_block_item(BlockSmem& sm, long long item_index, const float4* __restrict__ bodies,
                                               const SrcPair* __restrict__ pairs, const int4* __restrict__ items,
                                               const int2* __restrict__ item_rng, const int2* __restrict__ ranges,
                                               float4* __restrict__ near, int* __restrict__ err, const Lim& lim) {
  // the group partials of the final reduction reuse the first tile
  static_assert(sizeof(Acc<float>) * 2 * kThreads <= sizeof(SrcPair) * kTilePairs, "reduction space");
  SrcPair(*tiles)[kTilePairs] = sm.tiles;
  Stream& st = sm.st;
  unsigned long long* bar = sm.bar;
  int& abort_flag = sm.abort_flag;
  Acc<float>(*red)[kThreads] = reinterpret_cast<Acc<float>(*)[kThreads]>(&tiles[0][0]);
  // the item: targets [t0, t0 + nt) of the leaf with bodies [s, e) and
  // neighbour ranges [r0, r1)
  const int4 item = items[item_index];
  const int2 irng = item_rng[item_index];
  const int t0 = item.x, nt = item.y, s = item.z, e = item.w, r0 = irng.x, r1 = irng.y;
  const int tid = threadIdx.x;
  const f2 zero = make_float2(0.f, 0.f);
  if (tid == 0) {
    mbar_init(smem_u32(&bar[0]), 1);
    mbar_init(smem_u32(&bar[1]), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  const int nr = r1 - r0;
  const int nwin = (nr + kWindow - 1) / kWindow;
  int buf = 0;
  uint32_t parity = 0;  // bit b: the phase of bar[b] to wait for next
  {
    const int T2 = (nt + 1) >> 1;
    const int G = kThreads / T2;
    const int i = tid % T2, g = tid / T2;
    const bool active = g < G;
    const bool has_b = i + T2 < nt;
    f2 X0 = zero, Y0 = zero, Z0 = zero, X1 = zero, Y1 = zero, Z1 = zero;
    if (active) {
      const float4 a = GB_LD(bodies, t0 + i, lim.N, 106);
      const float4 b = has_b ? GB_LD(bodies, t0 + i + T2, lim.N, 106) : a;
      // negated, duplicated target coordinates
      X0 = f2_pack(-a.x, -a.x);
      Y0 = f2_pack(-a.y, -a.y);
      Z0 = f2_pack(-a.z, -a.z);
      X1 = f2_pack(-b.x, -b.x);
      Y1 = f2_pack(-b.y, -b.y);
      Z1 = f2_pack(-b.z, -b.z);
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
    // window -1: the leaf's own bodies (masked: self and coincident pairs
    // add zero); then the neighbour ranges, kWindow at a time
    for (int w = -1; w < nwin; ++w) {
      const int nw = w < 0 ? 1 : min(kWindow, nr - w * kWindow);
      if (tid < 32) {
        int P;
        if (w < 0) {
          const int ps = s >> 1, pe = (e + 1) >> 1;
          if (tid == 0) {
            st.rng[0] = make_int2(ps, (s & 1) | ((e & 1) << 1));
            st.pre[0] = 0;
            st.pre[1] = pe - ps;
          }
          P = pe - ps;
        } else {
          P = stage_window(st, ranges, r0 + w * kWindow, nw, lim);
        }
        if (tid == 0 && P > 0) mbar_arrive_expect_tx(smem_u32(&bar[buf]), (uint32_t)(min(P, kTilePairs) * sizeof(SrcPair)));
      }
      __syncthreads();
      const int P = st.pre[nw];
      const int ntile = (P + kTilePairs - 1) / kTilePairs;
      if (ntile > 0) {
        fence_async_smem();
        issue_tile(st, nw, 0, min(P, kTilePairs), pairs, smem_u32(tiles[buf]), smem_u32(&bar[buf]), lim);
      }
      for (int k = 0; k < ntile; ++k) {
        const int T0 = k * kTilePairs, T1 = min(T0 + kTilePairs, P);
        const uint32_t phase = (parity >> buf) & 1u;
        const bool ok = mbar_wait(smem_u32(&bar[buf]), phase, &abort_flag);
        parity ^= 1u << buf;
        if (ok) pad_tile(st, nw, T0, T1, tiles[buf]);
        const int T2n = min(T1 + kTilePairs, P);
        if (tid == 0 && T1 < P)
          mbar_arrive_expect_tx(smem_u32(&bar[buf ^ 1]), (uint32_t)((T2n - T1) * sizeof(SrcPair)));
        // the pads are visible and tiles[buf ^ 1] is no longer read
        if (__syncthreads_or(!ok)) {
          // a copy did not land in time: give up on this item.  The copies
          // of the tile waited for are the only ones in flight (the next
          // tile's are issued after this point); the block must not end
          // before they land in its shared memory, so thread 0 drains them
          // with a longer bounded wait.
          if (tid == 0) {
            atomicOr(err, kErrWait);
            if (!mbar_drain(smem_u32(&bar[buf]), phase)) atomicOr(err, kErrDrain);
          }
          return;
        }
        if (T1 < P) {
          fence_async_smem();
          issue_tile(st, nw, T1, T2n, pairs, smem_u32(tiles[buf ^ 1]), smem_u32(&bar[buf ^ 1]), lim);
        }
        if (active) {
          Acc2 p0{zero, zero, zero, zero}, p1{zero, zero, zero, zero};
          if (w < 0)
            tile_sum2<true>(tiles[buf], g, T1 - T0, G, X0, Y0, Z0, X1, Y1, Z1, p0, p1);
          else
            tile_sum2<false>(tiles[buf], g, T1 - T0, G, X0, Y0, Z0, X1, Y1, Z1, p0, p1);
          kahan_add(s0, c0, fold(p0));
          kahan_add(s1, c1, fold(p1));
        }
        buf ^= 1;
      }
      // the window's ranges and tiles are no longer read
      __syncthreads();
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
// Per-warp variant: each warp of a block owns one work item (a chunk of at
// most kWarpTargets targets of one leaf) and streams its sources through its
// own two shared-memory tiles, filled by bulk copies that complete on the
// warp's own mbarriers.  No block-wide barrier is needed: a warp waits only
// for its own copies, and its G groups (T2 targets each, two per lane) add
// their partial sums with shuffles at the end.
constexpr int kWarpTargets = 64;       // the per-warp code's limit (two targets per lane)
constexpr int kWarpSmallTargets = 16;  // items routed to it (measured: larger ones run faster per block)
constexpr int kWarpTile = 112;   // source pairs per warp tile (3.5 KB)
constexpr int kWarpWindow = 64;  // neighbour ranges staged at a time per warp
constexpr int kWarpsP2P = 4;

struct WStream {
  int2 rng[kWarpWindow];
  int pre[kWarpWindow + 1];
};

// Lane-strided forms of the block helpers above, for one warp.
__device__ __forceinline__ int stage_window_w(WStream& st, const int2* __restrict__ ranges, int r0, int nw,
                                              const Lim& lim, int lane) {
  int base = 0;
  for (int r = lane; r - lane < nw; r += 32) {
    int len = 0;
    if (r < nw) {
      const int2 rg = GB_LD(ranges, r0 + r, lim.nranges, 107);
      const int ps = rg.x >> 1, pe = (rg.y + 1) >> 1;
      st.rng[r] = make_int2(ps, (rg.x & 1) | ((rg.y & 1) << 1));
      len = pe - ps;
    }
    int incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (r < nw) st.pre[r] = base + incl - len;
    base += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) st.pre[nw] = base;
  return base;
}
__device__ __forceinline__ void issue_tile_w(const WStream& st, int nw, int T0, int T1,
                                             const SrcPair* __restrict__ src, uint32_t dst, uint32_t bar,
                                             const Lim& lim, int lane) {
  for (int r = lane; r < nw; r += 32) {
    const int pr = st.pre[r];
    const int a = max(pr, T0), b = min(st.pre[r + 1], T1);
    if (a < b) {
      const int first = st.rng[r].x + (a - pr);
#ifdef GBFMM_CHECKED
      if (!in_range(first + (b - a) - 1, (lim.N + 1) / 2, 108, lim.rec)) continue;
#endif
      bulk_g2s(dst + (uint32_t)(a - T0) * (uint32_t)sizeof(SrcPair), src + first,
               (uint32_t)(b - a) * (uint32_t)sizeof(SrcPair), bar);
    }
  }
}
__device__ __forceinline__ void pad_tile_w(const WStream& st, int nw, int T0, int T1, SrcPair* tile, int lane) {
  for (int r = lane; r < nw; r += 32) {
    const int f = st.rng[r].y;
    if (f == 0) continue;
    const int a = st.pre[r], b = st.pre[r + 1] - 1;
    if ((f & 1) && a >= T0 && a < T1) {
      tile[a - T0].w[0] = kFar;
      tile[a - T0].w[6] = 0.f;
    }
    if ((f & 2) && b >= T0 && b < T1) {
      tile[b - T0].w[1] = kFar;
      tile[b - T0].w[7] = 0.f;
    }
  }
}

// Shared memory of one block of the per-warp kernel.
struct WarpSmem {
  SrcPair tiles[kWarpsP2P][2][kWarpTile];
  WStream st[kWarpsP2P];
  unsigned long long bar[kWarpsP2P][2];
  int abort_w[kWarpsP2P];
};

// One work item per warp (the per-warp body of k_p2p_mix): items
// 4 wb .. 4 wb + 3 of `items` (nitem of them).
__device__ __forceinline__ void p2p_warp_items(WarpSmem& sm, long long wb, const float4* __restrict__ bodies,
                                               const SrcPair* __restrict__ pairs, const int4* __restrict__ items,
                                               const int2* __restrict__ item_rng, long long nitem,
                                               const int2* __restrict__ ranges, float4* __restrict__ near,
                                               int* __restrict__ err, const Lim& lim) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long it = wb * kWarpsP2P + warp;
  if (it >= nitem) return;  // the warp has no item (no block barrier follows)
  WStream& st = sm.st[warp];
  SrcPair(*tw)[kWarpTile] = sm.tiles[warp];
  const uint32_t bar0 = smem_u32(&sm.bar[warp][0]), bar1 = smem_u32(&sm.bar[warp][1]);
  volatile int* abort_flag = &sm.abort_w[warp];
  // the item: targets [t0, t0 + nt) of the leaf with bodies [s, e) and
  // neighbour ranges [r0, r1)
  const int4 item = items[it];
  const int2 irng = item_rng[it];
  const int t0 = item.x, nt = item.y, s = item.z, e = item.w, r0 = irng.x, r1 = irng.y;
  const f2 zero = make_float2(0.f, 0.f);
  if (lane == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar1, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncwarp();
  const int nr = r1 - r0;
  const int nwin = (nr + kWarpWindow - 1) / kWarpWindow;
  int buf = 0;
  uint32_t parity = 0;  // bit b: the phase of bar[b] to wait for next
  const int T2 = (nt + 1) >> 1;
  const int G = 32 / T2;
  const int i = lane % T2, g = lane / T2;
  const bool active = g < G;
  const bool has_b = i + T2 < nt;
  f2 X0 = zero, Y0 = zero, Z0 = zero, X1 = zero, Y1 = zero, Z1 = zero;
  if (active) {
    const float4 a = GB_LD(bodies, t0 + i, lim.N, 106);
    const float4 b = has_b ? GB_LD(bodies, t0 + i + T2, lim.N, 106) : a;
    // negated, duplicated target coordinates
    X0 = f2_pack(-a.x, -a.x);
    Y0 = f2_pack(-a.y, -a.y);
    Z0 = f2_pack(-a.z, -a.z);
    X1 = f2_pack(-b.x, -b.x);
    Y1 = f2_pack(-b.y, -b.y);
    Z1 = f2_pack(-b.z, -b.z);
  }
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
  bool failed = false;
  // window -1: the leaf's own bodies (masked: self and coincident pairs add
  // zero); then the neighbour ranges, kWarpWindow at a time
  for (int w = -1; w < nwin && !failed; ++w) {
    const int nw = w < 0 ? 1 : min(kWarpWindow, nr - w * kWarpWindow);
    int P;
    if (w < 0) {
      const int ps = s >> 1, pe = (e + 1) >> 1;
      if (lane == 0) {
        st.rng[0] = make_int2(ps, (s & 1) | ((e & 1) << 1));
        st.pre[0] = 0;
        st.pre[1] = pe - ps;
      }
      P = pe - ps;
    } else {
      P = stage_window_w(st, ranges, r0 + w * kWarpWindow, nw, lim, lane);
    }
    const int ntile = (P + kWarpTile - 1) / kWarpTile;
    if (lane == 0 && P > 0)
      mbar_arrive_expect_tx(buf ? bar1 : bar0, (uint32_t)(min(P, kWarpTile) * sizeof(SrcPair)));
    __syncwarp();  // the window's ranges are visible to the warp
    if (ntile > 0) {
      fence_async_smem();
      issue_tile_w(st, nw, 0, min(P, kWarpTile), pairs, smem_u32(tw[buf]), buf ? bar1 : bar0, lim, lane);
    }
    for (int k = 0; k < ntile; ++k) {
      const int T0 = k * kWarpTile, T1 = min(T0 + kWarpTile, P);
      const uint32_t phase = (parity >> buf) & 1u;
      const uint32_t mb = buf ? bar1 : bar0;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(mb, phase, abort_flag));
      parity ^= 1u << buf;
      if (!ok) {
        // a copy did not land in time: give up on this item after draining
        // the copies of the tile waited for (the only ones in flight)
        if (lane == 0) {
          atomicOr(err, kErrWait);
          if (!mbar_drain(mb, phase)) atomicOr(err, kErrDrain);
        }
        failed = true;
        break;
      }
      pad_tile_w(st, nw, T0, T1, tw[buf], lane);
      const int T2n = min(T1 + kWarpTile, P);
      if (lane == 0 && T1 < P)
        mbar_arrive_expect_tx(buf ? bar0 : bar1, (uint32_t)((T2n - T1) * sizeof(SrcPair)));
      __syncwarp();  // the pads are visible and tw[buf ^ 1] is no longer read
      if (T1 < P) {
        fence_async_smem();
        issue_tile_w(st, nw, T1, T2n, pairs, smem_u32(tw[buf ^ 1]), buf ? bar0 : bar1, lim, lane);
      }
      if (active) {
        Acc2 p0{zero, zero, zero, zero}, p1{zero, zero, zero, zero};
        if (w < 0)
          tile_sum2<true>(tw[buf], g, T1 - T0, G, X0, Y0, Z0, X1, Y1, Z1, p0, p1);
        else
          tile_sum2<false>(tw[buf], g, T1 - T0, G, X0, Y0, Z0, X1, Y1, Z1, p0, p1);
        kahan_add(s0, c0, fold(p0));
        kahan_add(s1, c1, fold(p1));
      }
      buf ^= 1;
    }
    __syncwarp();  // the window's ranges and tiles are no longer read
  }
  if (failed) return;
  // the G groups' partial sums, added in group order (reproducible)
  Acc<float> ta = s0, tb = s1;
  for (int gg = 1; gg < G; ++gg) {
    const int src_lane = gg * T2 + i;
    Acc<float> va, vb;
    va.p = __shfl_sync(0xffffffffu, s0.p, src_lane);
    va.x = __shfl_sync(0xffffffffu, s0.x, src_lane);
    va.y = __shfl_sync(0xffffffffu, s0.y, src_lane);
    va.z = __shfl_sync(0xffffffffu, s0.z, src_lane);
    vb.p = __shfl_sync(0xffffffffu, s1.p, src_lane);
    vb.x = __shfl_sync(0xffffffffu, s1.x, src_lane);
    vb.y = __shfl_sync(0xffffffffu, s1.y, src_lane);
    vb.z = __shfl_sync(0xffffffffu, s1.z, src_lane);
    ta.p += va.p; ta.x += va.x; ta.y += va.y; ta.z += va.z;
    tb.p += vb.p; tb.x += vb.x; tb.y += vb.y; tb.z += vb.z;
  }
  if (g == 0 && active) {
    GB_ST(near, t0 + i, lim.N, 109, make_float4(ta.p, ta.x, ta.y, ta.z));
    if (has_b) GB_ST(near, t0 + i + T2, lim.N, 109, make_float4(tb.p, tb.x, tb.y, tb.z));
  }
}

// The single-precision near field in one launch: blocks 0 .. nbig - 1 take one
// item each (items with many targets or sources), the blocks after them four
// items each, one per warp (items[nbig ..]).  Both parts share the block's
// shared memory; lower block indices are dispatched first, so the many short
// per-warp items fill the end of the per-block items.  Seven blocks per SM
// (at most 73 registers a thread): the pair chains are latency-bound, so
// resident warps count for more than a few spilled values.
union P2PSmem {
  BlockSmem b;
  WarpSmem w;
};

__global__ void __launch_bounds__(kThreads, 7) k_p2p_mix(const float4* __restrict__ bodies,
                                                      const SrcPair* __restrict__ pairs,
                                                      const int4* __restrict__ items,
                                                      const int2* __restrict__ item_rng, long long nbig,
                                                      long long nsmall, const int2* __restrict__ ranges,
                                                      float4* __restrict__ near, int* __restrict__ err, Lim lim) {
  __shared__ __align__(16) P2PSmem sm;
  if ((long long)blockIdx.x < nbig)
    p2p_block_item(sm.b, blockIdx.x, bodies, pairs, items, item_rng, ranges, near, err, lim);
  else
    p2p_warp_items(sm.w, (long long)blockIdx.x - nbig, bodies, pairs, items + nbig, item_rng + nbig, nsmall,
                   ranges, near, err, lim);
}

// Work items of the single-precision near field: a chunk of at most
// kItemTargets targets of one leaf, with the leaf's bodies (its own source
// range) and its neighbour ranges.  Per leaf, ceil(n / kItemTargets) chunks.
// Items are ordered by decreasing work (targets x sources), and block b
// takes item b: the block scheduler starts the largest first, which keeps
// the last wave short on workloads with a few large leaves.
constexpr int kItemTargets = kTgtChunk;
__global__ void k_item_count(const int32_t* __restrict__ leaves, const int32_t* __restrict__ bbeg,
                             const int32_t* __restrict__ bend, int nleaf, int per, int64_t* __restrict__ cnt) {
  const int li = blockIdx.x * blockDim.x + threadIdx.x;
  if (li > nleaf) return;
  if (li == nleaf) {
    cnt[li] = 0;
    return;
  }
  const int c = leaves[li];
  cnt[li] = (bend[c] - bbeg[c] + per - 1) / per;
}

// Sort key of an item: its work (targets x sources) in a 16-bit floating
// form (6-bit exponent, 10-bit mantissa; monotone in the work), inverted so
// that an ascending sort puts the largest first; bit 16 marks an item small
// enough for the per-warp kernel, so that the items of the per-block kernel
// come first.  Padding slots take the largest key.
constexpr int kWorkBits = 16;
constexpr int kKeyBits = kWorkBits + 1;
__device__ __forceinline__ uint64_t work_key(uint64_t work) {
  if (work == 0) return (1ull << kWorkBits) - 1;  // (an item always has targets and sources)
  const int e = 63 - __clzll((long long)work);  // work < 2^63
  const uint64_t m = (e >= 10 ? work >> (e - 10) : work << (10 - e)) & 0x3ffull;
  return ((1ull << kWorkBits) - 1) - ((uint64_t)(e + 1) << 10 | m);
}

__global__ void k_item_fill(const int32_t* __restrict__ leaves, const int32_t* __restrict__ bbeg,
                            const int32_t* __restrict__ bend, const int32_t* __restrict__ rptr,
                            const int2* __restrict__ ranges, int nleaf, int per, int warp_src,
                            const int64_t* __restrict__ ptr, int4* __restrict__ items, int2* __restrict__ rng,
                            uint64_t* __restrict__ key, int32_t* __restrict__ val,
                            unsigned long long* __restrict__ nbig) {
  const int li = blockIdx.x * blockDim.x + threadIdx.x;
  if (li >= nleaf) return;
  const int c = leaves[li];
  const int s = bbeg[c], e = bend[c], r0 = rptr[li], r1 = rptr[li + 1];
  long long src = e - s;
  for (int r = r0; r < r1; ++r) src += ranges[r].y - ranges[r].x;
  const int64_t p0 = ptr[li];
  for (int k = 0; s + k * per < e; ++k) {
    const int t0 = s + k * per, nt = min(per, e - t0);
    const int64_t idx = p0 + k;
    items[idx] = make_int4(t0, nt, s, e);
    rng[idx] = make_int2(r0, r1);
    const uint64_t work = (uint64_t)nt * (uint64_t)src;
    // the per-block code splits every tile among 128 / ceil(nt / 2) thread
    // groups, so on items with few targets and few sources its fixed costs
    // (block barriers per tile, the groups' reduction) outweigh the pairs:
    // those go to one warp each, whose smaller tiles cost more on long
    // source lists
    const bool small = nt <= kWarpSmallTargets && src <= warp_src;
    key[idx] = work_key(work) | (small ? 1ull << kWorkBits : 0ull);
    val[idx] = (int32_t)idx;
    if (!small) atomicAdd(nbig, 1ull);
  }
}

__global__ void k_item_pad(const int64_t* __restrict__ total, int64_t nmax, uint64_t* __restrict__ key,
                           int32_t* __restrict__ val) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= nmax || k < *total) return;
  key[k] = (1ull << kKeyBits) - 1;
  val[k] = (int32_t)k;
}

__global__ void k_item_gather(const int32_t* __restrict__ order, int64_t nmax, const int4* __restrict__ items_in,
                              const int2* __restrict__ rng_in, int4* __restrict__ items, int2* __restrict__ rng) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= nmax) return;
  items[k] = items_in[order[k]];
  rng[k] = rng_in[order[k]];
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

// Work items of at most kWarpSmallTargets targets and this many sources (the
// leaf's own bodies included) go to the per-warp code, the others to the
// per-block code (GBFMM_P2P_WARP_SRC: a tuning knob).
int p2p_warp_src() {
  static const int v = [] {
    const char* env = getenv("GBFMM_P2P_WARP_SRC");
    const int x = env ? atoi(env) : 2048;
    return x < 0 ? 0 : x;
  }();
  return v;
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
    const long long npair = (t->N + 1) / 2;
    k_pair_bodies<<<(unsigned)((npair + 255) / 256), 256, 0, s>>>((const float4*)t->work, t->N,
                                                                  (SrcPair*)t->near_src);
    GB_LAUNCH("k_pair_bodies");
    // items of more than the warp kernel's target limit: one per block;
    // the rest (after them in the list): one per warp
    const long long nbig = t->p2p_nbig_host, nsmall = t->p2p_nitem_host - nbig;
    const long long nblk = nbig + (nsmall + kWarpsP2P - 1) / kWarpsP2P;
    if (nblk > 0) {
      k_p2p_mix<<<(unsigned)nblk, kThreads, 0, s>>>((const float4*)t->work, (const SrcPair*)t->near_src,
                                                    t->p2p_items, t->p2p_item_rng, nbig, nsmall, t->p2p_ranges,
                                                    (float4*)t->near, t->dev_err, t->lim);
      GB_LAUNCH("k_p2p_mix");
    }
    return;
  }
  k_p2p<R, R4><<<t->nleaf, kThreads, 0, s>>>((const R4*)t->work, t->leaves, t->c.bbeg, t->c.bend, t->p2p_rptr,
                                             t->p2p_ranges, (R4*)t->near, t->lim);
  GB_LAUNCH("k_p2p");
}

// Near-field work items of the single-precision kernel, largest first (no
// host synchronisation: the item count stays in device memory and the arrays
// are sized by its bound nleaf + N / kItemTargets).
void build_p2p_items(fmm_tree* t) {
  Arena& a = t->arena;
  cudaStream_t s = t->stream;
  const int nleaf = (int)t->nleaf;
  const int per = kItemTargets;
  const int64_t nmax = (int64_t)nleaf + t->N / per + 1;
  const unsigned bl = (unsigned)((nleaf + 1 + 255) / 256), bm = (unsigned)((nmax + 255) / 256);
  int64_t* ptr = alloc_n<int64_t>(a, nleaf + 1);
  k_item_count<<<bl, 256, 0, s>>>(t->leaves, t->c.bbeg, t->c.bend, nleaf, per, ptr);
  GB_LAUNCH("k_item_count");
  t->p2p_nitem = alloc_n<long long>(a, 2);  // item count, then the count of per-block items
  GB_CK(cudaMemsetAsync(t->p2p_nitem + 1, 0, sizeof(long long), s));
  scan_exclusive_i64_dev(a, ptr, nleaf + 1, (int64_t*)t->p2p_nitem, s);
  int4* items = alloc_n<int4>(a, nmax);
  int2* rng = alloc_n<int2>(a, nmax);
  uint64_t* key = alloc_n<uint64_t>(a, nmax);
  int32_t* val = alloc_n<int32_t>(a, nmax);
  k_item_fill<<<bl, 256, 0, s>>>(t->leaves, t->c.bbeg, t->c.bend, t->p2p_rptr, t->p2p_ranges, nleaf, per,
                                 p2p_warp_src(), ptr, items, rng, key, val,
                                 reinterpret_cast<unsigned long long*>(t->p2p_nitem + 1));
  GB_LAUNCH("k_item_fill");
  k_item_pad<<<bm, 256, 0, s>>>((const int64_t*)t->p2p_nitem, nmax, key, val);
  GB_LAUNCH("k_item_pad");
  radix_sort_pairs(a, key, val, nmax, kKeyBits, s);
  t->p2p_items = alloc_n<int4>(a, nmax);
  t->p2p_item_rng = alloc_n<int2>(a, nmax);
  k_item_gather<<<bm, 256, 0, s>>>(val, nmax, items, rng, t->p2p_items, t->p2p_item_rng);
  GB_LAUNCH("k_item_gather");
  t->p2p_nitem_max = nmax;
  a.release(key);
  a.release(val);
  a.release(items);
  a.release(rng);
  a.release(ptr);
}

template void launch_p2p<float>(fmm_tree*, cudaStream_t);
template void launch_p2p<double>(fmm_tree*, cudaStream_t);

}  // namespace gbfmm
