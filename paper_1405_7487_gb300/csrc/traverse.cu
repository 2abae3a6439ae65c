// traverse.cu -- dual tree traversal into explicit P2P and M2L lists.
//
// The paper's ExaFMM finds M2L and P2P interactions by a dual tree traversal
// (Dehnen) without forming lists (Sec. II.C).  On the GPU the traversal runs
// breadth first over a frontier of unordered cell pairs and records the
// interactions as lists, which the evaluation and the backward pass reuse.
// Rules for a pair {A, B}:
//   A == B: a leaf takes P2P with itself; otherwise every unordered pair of
//           its children joins the next frontier.
//   MAC  theta |c_A - c_B| > R_A + R_B  (the bigger the cells, the further
//           apart they must be; Sec. II.A): M2L both ways.
//   two leaves: P2P both ways.
//   otherwise: split the larger cell (smaller level) unless it is a leaf, in
//           which case split the other; equal sizes, both split-table: every
//           (child of A, child of B) pair.
// The MAC is evaluated on exact integers (cube centres and radii in units of
// H / 2^21), so the lists are reproducible bit for bit.  With
// FMM_FLAG_TIGHT_MAC a cell's radius is instead the distance from its centre
// to its farthest body (the particle-fitted bound of Sec. II.B, the centre
// kept): its square is an exact integer over the bodies' 21-bit coordinates,
// and the test is theta^2 D^2 > (sqrt(r2_A) + sqrt(r2_B))^2 in correctly
// rounded double operations, the same on every device.  With
// FMM_FLAG_FITTED_CENTRES the centres move as well: to the centre of the box
// of the cell's voxel centres, an integer u_min + u_max + 1 per axis in the
// same units, and the radius is measured from there.
#include <algorithm>
#include <climits>
#include <cstdlib>

#include "common.cuh"
#include "grid.cuh"

namespace gbfmm {
namespace {

constexpr int kThreads = 256;
inline unsigned blocks(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

struct CellView {
  const int32_t *level, *ix, *iy, *iz, *cbeg, *nch;
  const double* rr;     // particle-fitted radius (tight MAC or fitted centres): the correctly rounded
                        // square root of its exact integer square, per cell, else null
  const int32_t* fc;    // fitted centres: 3 integer coordinates per cell (units H / 2^21), else null
};

__device__ __forceinline__ bool mac(const CellView& c, int A, int B, double theta2, int circ) {
  const int la = c.level[A], lb = c.level[B];
  const int64_t dx = ((2ll * c.ix[A] + 1) << (kMaxLevel - la)) - ((2ll * c.ix[B] + 1) << (kMaxLevel - lb));
  const int64_t dy = ((2ll * c.iy[A] + 1) << (kMaxLevel - la)) - ((2ll * c.iy[B] + 1) << (kMaxLevel - lb));
  const int64_t dz = ((2ll * c.iz[A] + 1) << (kMaxLevel - la)) - ((2ll * c.iz[B] + 1) << (kMaxLevel - lb));
  int64_t D2 = dx * dx + dy * dy + dz * dz;
  if (c.fc) {
    const int64_t fx = (int64_t)c.fc[3 * A] - c.fc[3 * B], fy = (int64_t)c.fc[3 * A + 1] - c.fc[3 * B + 1],
                  fz = (int64_t)c.fc[3 * A + 2] - c.fc[3 * B + 2];
    D2 = fx * fx + fy * fy + fz * fz;
  }
  if (c.rr) {
    const double sr = __dadd_rn(c.rr[A], c.rr[B]);
    return __dmul_rn(theta2, (double)D2) > __dmul_rn(sr, sr);
  }
  const int64_t rs = (1ll << (kMaxLevel - la)) + (1ll << (kMaxLevel - lb));
  int64_t S2 = rs * rs;
  if (circ) S2 *= 3;
  return __dmul_rn(theta2, (double)D2) > (double)S2;
}

// Decision for one pair: kind 0 = self leaf P2P, 1 = self split, 2 = M2L,
// 3 = P2P both ways, 4 = split A, 5 = split B, 6 = split both.
__device__ __forceinline__ int decide(const CellView& c, int A, int B, double theta2, int circ) {
  if (A == B) return c.nch[A] == 0 ? 0 : 1;
  if (mac(c, A, B, theta2, circ)) return 2;
  const bool la = c.nch[A] == 0, lb = c.nch[B] == 0;
  if (la && lb) return 3;
  if (c.level[A] < c.level[B]) return la ? 5 : 4;
  if (c.level[B] < c.level[A]) return lb ? 4 : 5;
  if (!la && !lb) return 6;
  return la ? 5 : 4;
}

// The (next, M2L, P2P) counts of one pair.
__device__ __forceinline__ void pair_counts(const CellView& c, int A, int B, int k, int& nn, int& nm, int& np) {
  nn = nm = np = 0;
  switch (k) {
    case 0: np = 1; break;
    case 1: nn = c.nch[A] * (c.nch[A] + 1) / 2; break;
    case 2: nm = 2; break;
    case 3: np = 2; break;
    case 4: nn = c.nch[A]; break;
    case 5: nn = c.nch[B]; break;
    default: nn = c.nch[A] * c.nch[B]; break;
  }
}

// Exclusive prefix of three per-thread counts over the block (kThreads
// threads, in thread order); the block's totals in tot.
__device__ __forceinline__ void block_scan3(int v[3], int tot[3]) {
  __shared__ int ws[3][kThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int inc[3] = {v[0], v[1], v[2]};
#pragma unroll
  for (int j = 0; j < 3; ++j)
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, inc[j], o);
      if (lane >= o) inc[j] += u;
    }
  if (lane == 31)
    for (int j = 0; j < 3; ++j) ws[j][w] = inc[j];
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    int before = 0, all = 0;
    for (int q = 0; q < kThreads / 32; ++q) {
      before += q < w ? ws[j][q] : 0;
      all += ws[j][q];
    }
    v[j] = before + inc[j] - v[j];
    tot[j] = all;
  }
  __syncthreads();  // ws is free for the next call
}

// Per block of frontier pairs: the totals of the three outputs, segment-major
// (cnt[j * nb + block]), so that one exclusive scan gives every block's
// output offsets in frontier order.
__global__ void __launch_bounds__(kThreads) k_trav_count(const int2* __restrict__ fr, int64_t n, CellView c,
                                                         double theta2, int circ, int64_t* __restrict__ cnt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int v[3] = {0, 0, 0}, tot[3];
  if (i < n) {
    const int A = fr[i].x, B = fr[i].y;
    pair_counts(c, A, B, decide(c, A, B, theta2, circ), v[0], v[1], v[2]);
  }
  block_scan3(v, tot);
  if (threadIdx.x == 0)
    for (int j = 0; j < 3; ++j) cnt[(int64_t)j * gridDim.x + blockIdx.x] = tot[j];
}

// A directed pair list as two arrays (target, source).
struct PairList {
  int32_t *tgt, *src;
  __device__ __forceinline__ void put(int64_t i, int t, int sr) const {
    tgt[i] = t;
    src[i] = sr;
  }
};

__device__ __forceinline__ uint64_t pair_key(int tgt, int src) {
  return ((uint64_t)(uint32_t)tgt << 32) | (uint32_t)src;
}

// M2L pair {A, B}: marks both cells as M2L cells and returns the largest |offset| component in units of the
// smaller cell's half side (the class offsets of the plan).  w[0] and w[1]
// receive the packed class offsets of the entries (target B, source A) and
// (target A, source B): bits 24..29 the level difference (source minus
// target) + 32, then the offset (source centre minus target centre) per
// axis as an 8-bit two's complement value, valid while every offset of the
// tree stays within +-127.
__device__ __forceinline__ unsigned mark_m2l(const CellView& c, int A, int B, int32_t* __restrict__ m2l_has,
                                             uint32_t w[2]) {
  const int la = c.level[A], lb = c.level[B], sh = kMaxLevel - (la > lb ? la : lb);
  const int co[2][3] = {{c.ix[A], c.iy[A], c.iz[A]}, {c.ix[B], c.iy[B], c.iz[B]}};
  unsigned dm = 0;
  w[0] = (uint32_t)(la - lb + 32) << 24;
  w[1] = (uint32_t)(lb - la + 32) << 24;
  for (int d = 0; d < 3; ++d) {
    const int64_t o = (((2ll * co[0][d] + 1) << (kMaxLevel - la)) - ((2ll * co[1][d] + 1) << (kMaxLevel - lb))) >> sh;
    dm = max(dm, (unsigned)(o < 0 ? -o : o));
    w[0] |= ((uint32_t)o & 0xffu) << (16 - 8 * d);
    w[1] |= ((uint32_t)(-o) & 0xffu) << (16 - 8 * d);
  }
  // per target, which level differences (source minus target: below, equal,
  // above) its M2L sources have, as bits 0, 1, 2 (read first)
  const int bitA = 1 << (lb < la ? 0 : (lb == la ? 1 : 2)), bitB = 1 << (la < lb ? 0 : (la == lb ? 1 : 2));
  if (!(m2l_has[A] & bitA)) atomicOr(m2l_has + A, bitA);
  if (!(m2l_has[B] & bitB)) atomicOr(m2l_has + B, bitB);
  return dm;
}

// The outputs of pair {A, B} (decision k) at next[o..], m2l[om..], p2p[op..].
__device__ __forceinline__ void write_pair(const CellView& c, int A, int B, int k, int64_t o, int64_t om, int64_t op,
                                           int2* __restrict__ next, PairList m2l, PairList p2p,
                                           uint32_t* __restrict__ m2l_off,
                                           const uint32_t w[2]) {
  switch (k) {
    case 0: p2p.put(op, A, A); break;
    case 1: {
      const int a0 = c.cbeg[A], na = c.nch[A];
      for (int x = 0; x < na; ++x)
        for (int y = x; y < na; ++y) next[o++] = make_int2(a0 + x, a0 + y);
      break;
    }
    case 2:
      m2l.put(om, B, A);
      m2l.put(om + 1, A, B);
      m2l_off[om] = w[0];
      m2l_off[om + 1] = w[1];
      break;
    case 3:
      p2p.put(op, B, A);
      p2p.put(op + 1, A, B);
      break;
    case 4: {
      const int a0 = c.cbeg[A], na = c.nch[A];
      for (int x = 0; x < na; ++x) next[o++] = make_int2(a0 + x, B);
      break;
    }
    case 5: {
      const int b0 = c.cbeg[B], nb = c.nch[B];
      for (int y = 0; y < nb; ++y) next[o++] = make_int2(A, b0 + y);
      break;
    }
    default: {
      const int a0 = c.cbeg[A], na = c.nch[A], b0 = c.cbeg[B], nb = c.nch[B];
      for (int x = 0; x < na; ++x)
        for (int y = 0; y < nb; ++y) next[o++] = make_int2(a0 + x, b0 + y);
      break;
    }
  }
}

// The largest class offset of the block's M2L pairs into *m2l_maxd (read
// first: most blocks find it already as large).
__device__ __forceinline__ void block_maxd(unsigned dm, unsigned long long* __restrict__ m2l_maxd) {
  __shared__ unsigned wmax[kThreads / 32];
  dm = __reduce_max_sync(0xffffffffu, dm);
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = dm;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kThreads / 32; ++w) dm = max(dm, wmax[w]);
    if (dm > *(volatile unsigned long long*)m2l_maxd) atomicMax(m2l_maxd, (unsigned long long)dm);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads) k_trav_write(const int2* __restrict__ fr, int64_t n, CellView c,
                                                         double theta2, int circ, const int64_t* __restrict__ off,
                                                         int64_t base_m, int64_t base_p, int2* __restrict__ next,
                                                         PairList m2l, int64_t m2l_at, PairList p2p,
                                                         int64_t p2p_at,
                                                         int32_t* __restrict__ m2l_has,
                                                         unsigned long long* __restrict__ m2l_maxd,
                                                         uint32_t* __restrict__ m2l_off) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int A = 0, B = 0, k = -1, v[3] = {0, 0, 0}, tot[3];
  unsigned dm = 0;
  uint32_t w[2] = {0, 0};
  if (i < n) {
    A = fr[i].x;
    B = fr[i].y;
    k = decide(c, A, B, theta2, circ);
    pair_counts(c, A, B, k, v[0], v[1], v[2]);
    if (k == 2) dm = mark_m2l(c, A, B, m2l_has, w);
  }
  block_scan3(v, tot);
  block_maxd(dm, m2l_maxd);
  if (i >= n) return;
  const int nb = gridDim.x;
  write_pair(c, A, B, k, off[blockIdx.x] + v[0], m2l_at + off[nb + blockIdx.x] - base_m + v[1],
             p2p_at + off[2 * nb + blockIdx.x] - base_p + v[2], next, m2l, p2p, m2l_off, w);
}

// The whole traversal in one cooperative launch, while the frontier and the
// lists fit the buffers given (capF pairs per frontier, cap_m and cap_p list
// entries).  Each level splits the frontier into contiguous chunks, one per
// block: the blocks count their outputs, publish the three totals and, after
// a grid barrier, add the totals of the blocks before them and write, so the
// outputs come in frontier order, as with the per-level launches.  The next
// frontier alternates between F0 and F1 (read through L2: other blocks wrote
// it).  If a level would overflow a buffer every block stops before writing
// it and st->overflow is set.
struct TravState {
  long long nm, np, ntgt;  // M2L and P2P entries, cells that take M2L
  int nlevel, overflow;
  GridBar bar;
};

// Cells flagged in has[0 .. n) into *count (read through L2: the flags were
// set by other blocks of the launch, or by an earlier launch).
__device__ __forceinline__ void count_flags(const int32_t* has, int64_t n, long long* count) {
  __shared__ long long wsum[kThreads / 32];
  long long c = 0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
    c += __ldcg(has + i) != 0;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kThreads / 32; ++w) c += wsum[w];
    if (c) atomicAdd(reinterpret_cast<unsigned long long*>(count), (unsigned long long)c);
  }
}

__global__ void __launch_bounds__(kThreads) k_count_flags(const int32_t* __restrict__ has, int64_t n,
                                                          TravState* __restrict__ st) {
  count_flags(has, n, &st->ntgt);
}

__global__ void __launch_bounds__(kThreads) k_traverse(CellView c, int ncell, double theta2, int circ, int2* F0,
                                                       int2* F1,
                                                       long long capF, PairList m2l, long long cap_m, PairList p2p,
                                                       long long cap_p,
                                                       int32_t* __restrict__ m2l_has,
                                                       unsigned long long* __restrict__ m2l_maxd,
                                                       uint32_t* __restrict__ m2l_off, int2* __restrict__ info,
                                                       const int32_t* __restrict__ leaf_of,
                                                       const int32_t* __restrict__ bbeg,
                                                       const int32_t* __restrict__ bend, int64_t* __restrict__ leaf_cnt,
                                                       unsigned long long* __restrict__ body_pairs,
                                                       long long* __restrict__ partial, TravState* st,
                                                       int* __restrict__ err) {
  const int G = gridDim.x, blk = blockIdx.x;
  if (blk == 0 && threadIdx.x == 0) F0[0] = make_int2(0, 0);
  int2 *cur = F0, *nxt = F1;
  long long nf = 1, nm = 0, np = 0;
  int nlevel = 0;
  unsigned dm = 0;
  unsigned long long bp = 0;  // this thread's body pairs
  bool fine = grid_barrier(&st->bar, err), over = false;
  while (fine && nf > 0) {
    ++nlevel;
    const long long ch = (nf + G - 1) / G;
    const long long f0 = min(blk * ch, nf), f1 = min((blk + 1) * ch, nf);
    // count: the decision, the three counts and (M2L) the packed class offset
    // of each pair are kept in info[i] for the write pass, which then needs
    // no cell data but for splits
    long long cnt[3] = {0, 0, 0};
    for (long long i = f0 + threadIdx.x; i < f1; i += kThreads) {
      const int2 pr = __ldcg(cur + i);
      const int k = decide(c, pr.x, pr.y, theta2, circ);
      int v[3];
      pair_counts(c, pr.x, pr.y, k, v[0], v[1], v[2]);
      uint32_t w[2] = {0, 0};
      if (k == 2) dm = max(dm, mark_m2l(c, pr.x, pr.y, m2l_has, w));
      info[i] = make_int2(k | (v[0] << 3) | (v[1] << 10) | (v[2] << 12), (int)w[0]);
      for (int j = 0; j < 3; ++j) cnt[j] += v[j];
    }
    {
      __shared__ long long wc[3][kThreads / 32];
      for (int j = 0; j < 3; ++j)
        for (int o = 16; o > 0; o >>= 1) cnt[j] += __shfl_down_sync(0xffffffffu, cnt[j], o);
      if ((threadIdx.x & 31) == 0)
        for (int j = 0; j < 3; ++j) wc[j][threadIdx.x >> 5] = cnt[j];
      __syncthreads();
      if (threadIdx.x == 0)
        for (int j = 0; j < 3; ++j) {
          long long t = 0;
          for (int w = 0; w < kThreads / 32; ++w) t += wc[j][w];
          partial[(int64_t)j * G + blk] = t;
        }
    }
    fine = grid_barrier(&st->bar, err);
    if (!fine) break;
    long long before[3], total[3];
    block_prefix_totals<long long, 3>(partial, blk, G, before, total);
    if (total[0] > capF || nm + total[1] > cap_m || np + total[2] > cap_p) {  // the same in every block
      if (blk == 0 && threadIdx.x == 0) st->overflow = 1;
      over = true;
      break;
    }
    long long run[3] = {before[0], nm + before[1], np + before[2]};
    for (long long base = f0; base < f1; base += kThreads) {
      const long long i = base + threadIdx.x;
      int A = 0, B = 0, k = -1, v[3] = {0, 0, 0}, tot[3];
      uint32_t w[2] = {0, 0};
      if (i < f1) {
        const int2 pr = __ldcg(cur + i);
        const int2 in = info[i];
        A = pr.x;
        B = pr.y;
        k = in.x & 7;
        v[0] = (in.x >> 3) & 127;
        v[1] = (in.x >> 10) & 3;
        v[2] = (in.x >> 12) & 3;
        w[0] = (uint32_t)in.y;
        // the entry (target A, source B): level difference and offsets negated
        w[1] = (64u - (w[0] >> 24)) << 24;
        for (int d = 0; d < 3; ++d) w[1] |= ((uint32_t)(-(int)(int8_t)(w[0] >> (16 - 8 * d))) & 0xffu) << (16 - 8 * d);
      }
      block_scan3(v, tot);
      if (i < f1) {
        write_pair(c, A, B, k, run[0] + v[0], run[1] + v[1], run[2] + v[2], nxt, m2l, p2p, m2l_off, w);
        // P2P: each target leaf's count of sources (self excluded) and the body pairs
        if (k == 0) {
          const unsigned long long na = bend[A] - bbeg[A];
          bp += na * na;
        } else if (k == 3) {
          bp += 2ull * (unsigned long long)(bend[A] - bbeg[A]) * (unsigned long long)(bend[B] - bbeg[B]);
          atomicAdd(reinterpret_cast<unsigned long long*>(leaf_cnt + leaf_of[A]), 1ull);
          atomicAdd(reinterpret_cast<unsigned long long*>(leaf_cnt + leaf_of[B]), 1ull);
        }
      }
      for (int j = 0; j < 3; ++j) run[j] += tot[j];
    }
    fine = grid_barrier(&st->bar, err);
    int2* t = cur;
    cur = nxt;
    nxt = t;
    nf = total[0];
    nm += total[1];
    np += total[2];
  }
  if (!fine) return;
  block_maxd(dm, m2l_maxd);
  if (!over) {
    count_flags(m2l_has, ncell, &st->ntgt);
    for (int o = 16; o > 0; o >>= 1) bp += __shfl_down_sync(0xffffffffu, bp, o);
    if ((threadIdx.x & 31) == 0 && bp) atomicAdd(body_pairs, bp);
  }
  if (blk == 0 && threadIdx.x == 0 && !over) {
    st->nm = nm;
    st->np = np;
    st->nlevel = nlevel;
  }
}

__global__ void k_pack_pairs(const int32_t* __restrict__ tgt, const int32_t* __restrict__ src, int64_t n,
                             uint64_t* __restrict__ k) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) k[i] = ((uint64_t)(uint32_t)tgt[i] << 32) | (uint32_t)src[i];
}

__global__ void k_unpack_pairs(const uint64_t* __restrict__ k, int64_t n, int32_t* __restrict__ tgt,
                               int32_t* __restrict__ src) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  tgt[i] = (int32_t)(k[i] >> 32);
  src[i] = (int32_t)(k[i] & 0xffffffffu);
}

// P2P source lists by target leaf: a counting sort by leaf, then each leaf's
// sources in body order (their body ranges are disjoint, so the order is
// unique).  Count pass: non-self pairs per leaf, and the body-pair total.
__global__ void k_p2p_leaf_count(const int32_t* __restrict__ tgt, const int32_t* __restrict__ src, int64_t n,
                                 const int32_t* __restrict__ leaf_of, const int32_t* __restrict__ bbeg,
                                 const int32_t* __restrict__ bend, int64_t* __restrict__ cnt,
                                 unsigned long long* __restrict__ pairs) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  unsigned long long np = 0;
  if (i < n) np = (unsigned long long)(bend[tgt[i]] - bbeg[tgt[i]]) * (unsigned long long)(bend[src[i]] - bbeg[src[i]]);
  for (int o = 16; o > 0; o >>= 1) np += __shfl_down_sync(0xffffffffu, np, o);
  if ((threadIdx.x & 31) == 0 && np) atomicAdd(pairs, np);
  if (i < n && tgt[i] != src[i]) atomicAdd(reinterpret_cast<unsigned long long*>(&cnt[leaf_of[tgt[i]]]), 1ull);
}

__global__ void k_p2p_leaf_scatter(const int32_t* __restrict__ tgt, const int32_t* __restrict__ src, int64_t n,
                                   const int32_t* __restrict__ leaf_of, const int64_t* __restrict__ ptr,
                                   int32_t* __restrict__ cursor, int32_t* __restrict__ val) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n || tgt[i] == src[i]) return;
  const int l = leaf_of[tgt[i]];
  val[ptr[l] + atomicAdd(&cursor[l], 1)] = src[i];
}

// Each leaf's sources ordered by body begin, from `in` to `out` (the keys
// are distinct: the sources' body ranges are disjoint).  A block of four
// warps takes four leaves.  A list of at most kWarpRank entries is sorted by
// its warp: the keys go to the warp's part of shared memory and each entry's
// place is the number of smaller keys (every lane reads the same key at a
// time, so the reads are broadcasts).  Longer lists are sorted by the whole
// block, one after another: up to kSegSort entries a bitonic sort in shared
// memory, beyond that (none at the workloads here) each entry ranked by
// counting the smaller ones in global memory.
constexpr int kSegSort = 1024;
constexpr int kLeavesPerSortBlock = 4;
constexpr int kWarpRank = kSegSort / kLeavesPerSortBlock;
__device__ void sort_long_list(int64_t b, int L, const int32_t* __restrict__ bbeg, const int32_t* __restrict__ in,
                               int32_t* __restrict__ out, int* sk, int* sv) {
  if (L <= kSegSort) {
    int n2 = 1;
    while (n2 < L) n2 <<= 1;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) {
      const bool ok = i < L;
      const int v = ok ? in[b + i] : -1;
      sv[i] = v;
      sk[i] = ok ? bbeg[v] : INT_MAX;
    }
    __syncthreads();
    for (int k = 2; k <= n2; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < n2; i += blockDim.x) {
          const int x = i ^ j;
          if (x > i) {
            const bool up = (i & k) == 0;
            if ((sk[i] > sk[x]) == up) {
              const int tk = sk[i], tv = sv[i];
              sk[i] = sk[x];
              sv[i] = sv[x];
              sk[x] = tk;
              sv[x] = tv;
            }
          }
        }
        __syncthreads();
      }
    for (int i = threadIdx.x; i < L; i += blockDim.x) out[b + i] = sv[i];
  } else {
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
      const int v = in[b + i], key = bbeg[v];
      int r = 0;
      for (int j = 0; j < L; ++j) r += bbeg[in[b + j]] < key;
      out[b + r] = v;
    }
  }
}
__global__ void k_p2p_leaf_sort(const int64_t* __restrict__ ptr, int nleaf, const int32_t* __restrict__ bbeg,
                                const int32_t* __restrict__ in, int32_t* __restrict__ out) {
  __shared__ int sk[kSegSort], sv[kSegSort];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  {
    const int l = blockIdx.x * kLeavesPerSortBlock + w;
    if (l < nleaf) {
      const int64_t b = ptr[l];
      const int L = (int)(ptr[l + 1] - b);
      if (L <= kWarpRank) {
        int* k = sk + w * kWarpRank;
        int* v = sv + w * kWarpRank;
        for (int i = lane; i < L; i += 32) {
          const int x = in[b + i];
          v[i] = x;
          k[i] = bbeg[x];
        }
        __syncwarp();
        for (int i = lane; i < L; i += 32) {
          const int key = k[i];
          int r = 0;
          for (int j = 0; j < L; ++j) r += k[j] < key;
          out[b + r] = v[i];
        }
      }
    }
  }
  __syncthreads();
  for (int q = 0; q < kLeavesPerSortBlock; ++q) {
    const int l = blockIdx.x * kLeavesPerSortBlock + q;
    if (l >= nleaf) return;
    const int64_t b = ptr[l];
    const int L = (int)(ptr[l + 1] - b);
    if (L <= kWarpRank) continue;
    sort_long_list(b, L, bbeg, in, out, sk, sv);
    __syncthreads();
  }
}

// Merge adjacent body ranges of one target leaf (its sources in body order);
// count pass (out == null) or write pass.  A warp per leaf, 32 sources at a
// time: a source starts a merged range unless its body range begins where
// the previous one ended, and ends one unless the next begins where it ends.
constexpr int kMergeWarps = 8;
__global__ void __launch_bounds__(32 * kMergeWarps)
    k_merge_ranges(const int64_t* __restrict__ eptr, const int32_t* __restrict__ val,
                   const int32_t* __restrict__ bbeg, const int32_t* __restrict__ bend, int nleaf,
                   int64_t* __restrict__ count, const int64_t* __restrict__ out_off, int2* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int l = blockIdx.x * kMergeWarps + (threadIdx.x >> 5);
  if (l >= nleaf) return;
  const int64_t e0 = eptr[l], e1 = eptr[l + 1];
  const int64_t o = out ? out_off[l] : 0;
  int64_t runs = 0;  // merged ranges started before this group of 32
  int prev_end = -1;  // body end of the source before this group
  for (int64_t g = e0; g < e1; g += 32) {
    const int64_t e = g + lane;
    const bool ok = e < e1;
    int b = 0, en = 0, nb = -2;
    if (ok) {
      const int sr = val[e];
      b = bbeg[sr];
      en = bend[sr];
      if (e + 1 < e1) nb = bbeg[val[e + 1]];
    }
    int pe = __shfl_up_sync(0xffffffffu, en, 1);
    if (lane == 0) pe = prev_end;
    const bool start = ok && b != pe;
    const bool last = ok && nb != en;
    const unsigned sm = __ballot_sync(0xffffffffu, start);
    const int64_t k = runs + __popc(sm & ((2u << lane) - 1u)) - 1;  // this source's range
    if (out) {
      if (start) out[o + k].x = b;
      if (last) out[o + k].y = en;
    }
    runs += __popc(sm);
    prev_end = __shfl_sync(0xffffffffu, en, 31);
  }
  if (count && lane == 0) count[l] = runs;
}

__global__ void k_i64_to_i32(const int64_t* __restrict__ a, int64_t n, int32_t* __restrict__ b) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (int32_t)a[i];
}

// Mutual interaction: the unordered leaf pairs (source cell < target cell)
// of the symmetric P2P list.
__global__ void k_upair_flags(const int32_t* __restrict__ tgt, const int32_t* __restrict__ src, int64_t n,
                              int64_t* __restrict__ f) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) f[i] = src[i] < tgt[i] ? 1 : 0;
}

__global__ void k_upair_write(const int32_t* __restrict__ tgt, const int32_t* __restrict__ src, int64_t n,
                              const int64_t* __restrict__ off, int2* __restrict__ up) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n && src[i] < tgt[i]) up[off[i]] = make_int2(src[i], tgt[i]);
}

// Squared particle-fitted radius of every cell: the largest squared distance
// from the cell centre (2k + 1) 2^(21 - l) to a body's voxel centre 2u + 1,
// per axis in units of H / 2^21, u the body's 21-bit coordinate (read back
// from its sorted Morton key).  One block per cell.
__device__ __forceinline__ int64_t compact3(uint64_t v) {
  v &= 0x1249249249249249ull;
  v = (v | (v >> 2)) & 0x10c30c30c30c30c3ull;
  v = (v | (v >> 4)) & 0x100f00f00f00f00full;
  v = (v | (v >> 8)) & 0x1f0000ff0000ffull;
  v = (v | (v >> 16)) & 0x1f00000000ffffull;
  v = (v | (v >> 32)) & 0x1fffffull;
  return (int64_t)v;
}

__global__ void k_cell_r2(const uint64_t* __restrict__ keys, const int32_t* __restrict__ level,
                          const int32_t* __restrict__ ix, const int32_t* __restrict__ iy,
                          const int32_t* __restrict__ iz, const int32_t* __restrict__ bbeg,
                          const int32_t* __restrict__ bend, long long* __restrict__ r2) {
  const int c = blockIdx.x;
  const int sh = kMaxLevel - level[c];
  const int64_t cx = (2ll * ix[c] + 1) << sh, cy = (2ll * iy[c] + 1) << sh, cz = (2ll * iz[c] + 1) << sh;
  long long m = 0;
  for (int i = bbeg[c] + threadIdx.x; i < bend[c]; i += blockDim.x) {
    const uint64_t k = keys[i];
    const int64_t dx = 2 * compact3(k >> 2) + 1 - cx, dy = 2 * compact3(k >> 1) + 1 - cy, dz = 2 * compact3(k) + 1 - cz;
    m = max(m, (long long)(dx * dx + dy * dy + dz * dz));
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
  __shared__ long long wm[32];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = max(m, wm[w]);
    r2[c] = m;
  }
}

// Fitted centres: per cell the box of its bodies' voxel centres 2u + 1 (u
// their 21-bit coordinates, read back from the sorted keys), its centre
// u_min + u_max + 1 per axis and the squared distance from there to the
// farthest voxel centre, all exact integers in units of H / 2^21.  One block
// per cell.
__global__ void k_cell_fit(const uint64_t* __restrict__ keys, const int32_t* __restrict__ bbeg,
                           const int32_t* __restrict__ bend, int32_t* __restrict__ fc, long long* __restrict__ r2) {
  const int c = blockIdx.x;
  __shared__ int wl[3][32], wh[3][32];
  __shared__ int ctr[3];
  __shared__ long long wm[32];
  int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {-1, -1, -1};
  for (int i = bbeg[c] + threadIdx.x; i < bend[c]; i += blockDim.x) {
    const uint64_t k = keys[i];
    const int u[3] = {(int)compact3(k >> 2), (int)compact3(k >> 1), (int)compact3(k)};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      lo[a] = min(lo[a], u[a]);
      hi[a] = max(hi[a], u[a]);
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a)
    for (int o = 16; o > 0; o >>= 1) {
      lo[a] = min(lo[a], __shfl_down_sync(0xffffffffu, lo[a], o));
      hi[a] = max(hi[a], __shfl_down_sync(0xffffffffu, hi[a], o));
    }
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0)
    for (int a = 0; a < 3; ++a) {
      wl[a][w] = lo[a];
      wh[a][w] = hi[a];
    }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int a = 0; a < 3; ++a) {
      int l = wl[a][0], h = wh[a][0];
      for (int v = 1; v < nw; ++v) {
        l = min(l, wl[a][v]);
        h = max(h, wh[a][v]);
      }
      ctr[a] = l + h + 1;
      fc[3 * c + a] = ctr[a];
    }
  __syncthreads();
  long long m = 0;
  for (int i = bbeg[c] + threadIdx.x; i < bend[c]; i += blockDim.x) {
    const uint64_t k = keys[i];
    const int64_t dx = 2 * compact3(k >> 2) + 1 - ctr[0], dy = 2 * compact3(k >> 1) + 1 - ctr[1],
                  dz = 2 * compact3(k) + 1 - ctr[2];
    m = max(m, (long long)(dx * dx + dy * dy + dz * dz));
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wm[w] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int v = 1; v < nw; ++v) m = max(m, wm[v]);
    r2[c] = m;
  }
}

}  // namespace

// Smallest b with 2^b > v.
int bits_for(int64_t v) {
  int b = 0;
  while (b < 63 && (1ll << b) <= v) ++b;
  return b;
}

// (target, source) order of a directed pair list, for the inspection call.
void sort_pairs_copy(Arena& a, const int32_t* tgt, const int32_t* src, int64_t n, int ncell, int32_t* out_tgt,
                     int32_t* out_src, cudaStream_t s) {
  if (n == 0) return;
  uint64_t* k = alloc_n<uint64_t>(a, n);
  k_pack_pairs<<<blocks(n), kThreads, 0, s>>>(tgt, src, n, k);
  GB_LAUNCH("k_pack_pairs");
  radix_sort_keys(a, k, n, 32 + bits_for(ncell), s);
  k_unpack_pairs<<<blocks(n), kThreads, 0, s>>>(k, n, out_tgt, out_src);
  GB_LAUNCH("k_unpack_pairs");
  a.release(k);
}

__global__ void k_cell_root(const long long* __restrict__ r2, int n, double* __restrict__ rr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) rr[i] = __dsqrt_rn((double)r2[i]);
}

void build_lists(fmm_tree* t) {
  Arena& a = t->arena;
  cudaStream_t s = t->stream;
  long long* r2 = nullptr;
  if (t->flags & FMM_FLAG_FITTED_CENTRES) {
    // the integer centres stay with the tree (the expansion centres follow
    // from them)
    r2 = alloc_n<long long>(a, t->ncell);
    t->fit_c = alloc_n<int32_t>(a, 3 * (size_t)t->ncell);
    k_cell_fit<<<(unsigned)t->ncell, 128, 0, s>>>(t->keys, t->c.bbeg, t->c.bend, t->fit_c, r2);
    GB_LAUNCH("k_cell_fit");
  } else if (t->flags & FMM_FLAG_TIGHT_MAC) {
    r2 = alloc_n<long long>(a, t->ncell);
    k_cell_r2<<<(unsigned)t->ncell, 128, 0, s>>>(t->keys, t->c.level, t->c.ix, t->c.iy, t->c.iz, t->c.bbeg,
                                                t->c.bend, r2);
    GB_LAUNCH("k_cell_r2");
  }
  // the radii's square roots once per cell (the same doubles the per-pair
  // test took, without two FP64 square roots per candidate pair)
  double* rr = nullptr;
  if (r2) {
    rr = alloc_n<double>(a, t->ncell);
    k_cell_root<<<blocks(t->ncell), kThreads, 0, s>>>(r2, t->ncell, rr);
    GB_LAUNCH("k_cell_root");
  }
  CellView cv{t->c.level, t->c.ix, t->c.iy, t->c.iz, t->c.cbeg, t->c.nch, rr, t->fit_c};
  const double theta2 = t->theta * t->theta;
  const int circ = (t->flags & FMM_FLAG_CIRCUMSCRIBED) ? 1 : 0;

  // for the M2L plan: the cells that take M2L and the largest class offset
  t->m2l_has = alloc_n<int32_t>(a, t->ncell);
  t->m2l_maxd = alloc_n<unsigned long long>(a, 1);
  GB_CK(cudaMemsetAsync(t->m2l_has, 0, sizeof(int32_t) * t->ncell, s));
  GB_CK(cudaMemsetAsync(t->m2l_maxd, 0, sizeof(unsigned long long), s));

  // The whole traversal in one cooperative launch when the frontier and the
  // lists fit buffers of 64 N entries in all (two frontiers of a fifth each,
  // M2L half, P2P a tenth; the workloads here use at most about half of
  // each); then one read-back.  Otherwise the per-level launches below take
  // over, with one read-back per level (the marks already made are kept:
  // they are a subset of the final ones).
  // per target leaf its count of sources (then their offsets), and the body
  // pairs; the range count and the body-pair total stay on the device until
  // the end of the build (t->d_tail[0], t->d_tail[1])
  t->d_tail = alloc_n<long long>(a, 4);
  GB_CK(cudaMemsetAsync(t->d_tail, 0, 4 * sizeof(long long), s));
  unsigned long long* d_pairs = reinterpret_cast<unsigned long long*>(t->d_tail + 1);
  int64_t* eptr = alloc_n<int64_t>(a, t->nleaf + 1);
  GB_CK(cudaMemsetAsync(eptr, 0, sizeof(int64_t) * (t->nleaf + 1), s));
  // The MACs with true bounds (circumscribed, particle-fitted) accept fewer
  // pairs at the same theta: their lists run 3 to 6 times longer (92.6 M M2L
  // entries for 1 M Plummer bodies with fitted centres, against 25.7 M).
  const bool long_lists = (t->flags & (FMM_FLAG_CIRCUMSCRIBED | FMM_FLAG_TIGHT_MAC | FMM_FLAG_FITTED_CENTRES)) != 0;
  int64_t budget = std::max<int64_t>(1ll << 23, (long_lists ? 256 : 64) * t->N);
  // GBFMM_TRAVERSE_BUDGET (entries) overrides it: a small value makes the
  // single launch stop early and the per-level launches take over (the test
  // of that path)
  if (const char* env = getenv("GBFMM_TRAVERSE_BUDGET")) budget = std::max<int64_t>(16, atoll(env));
  int64_t cap_m = budget / 2, cap_p = budget / 10;
  const int64_t capF = budget / 5;
  // the lists are written in place and kept at this capacity (no copy)
  PairList m2l{alloc_n<int32_t>(a, cap_m), alloc_n<int32_t>(a, cap_m)};
  PairList p2p{alloc_n<int32_t>(a, cap_p), alloc_n<int32_t>(a, cap_p)};
  t->m2l_off = alloc_n<uint32_t>(a, cap_m);  // packed class offsets, kept for the plan
  int64_t nm = 0, np = 0;
  bool done = false;
  {
    int sms = 0, dev = 0, per_sm = 0;
    GB_CK(cudaGetDevice(&dev));
    GB_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    GB_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_traverse, kThreads, 0));
    const int G = std::max(1, std::min(4, per_sm) * sms);
    int2* F0 = alloc_n<int2>(a, capF);
    int2* F1 = alloc_n<int2>(a, capF);
    long long* partial = alloc_n<long long>(a, 3 * (size_t)G);
    TravState* d_st = alloc_n<TravState>(a, 1);
    int2* info = alloc_n<int2>(a, capF);
    GB_CK(cudaMemsetAsync(d_st, 0, sizeof(TravState), s));
    long long capF_ = capF, cap_m_ = cap_m, cap_p_ = cap_p;
    int* err = a.err;
    const int ncell = t->ncell;
    void* args[] = {(void*)&cv,     (void*)&ncell,  (void*)&theta2, (void*)&circ, (void*)&F0, (void*)&F1,
                    (void*)&capF_,  (void*)&m2l,    (void*)&cap_m_,     (void*)&p2p,        (void*)&cap_p_,
                    (void*)&t->m2l_has, (void*)&t->m2l_maxd, (void*)&t->m2l_off, (void*)&info,
                    (void*)&t->leaf_of_cell, (void*)&t->c.bbeg, (void*)&t->c.bend, (void*)&eptr, (void*)&d_pairs,
                    (void*)&partial, (void*)&d_st, (void*)&err};
    GB_CK(cudaLaunchCooperativeKernel((const void*)k_traverse, dim3(G), dim3(kThreads), args, 0, s));
    GB_LAUNCH("k_traverse");
    TravState h;
    GB_CK(cudaMemcpyAsync(&h, d_st, sizeof(TravState), cudaMemcpyDeviceToHost, s));
    GB_CK(cudaMemcpyAsync(&t->m2l_maxd_host, t->m2l_maxd, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    check_scan_error(a, s);  // synchronises; a grid wait past its limit is FMM_ERR_TIMEOUT
    if (!h.overflow) {
      nm = h.nm;
      np = h.np;
      t->m2l_ntgt = h.ntgt;
      done = true;
    }
    a.release(info);
    a.release(d_st);
    a.release(partial);
    a.release(F1);
    a.release(F0);
  }
  if (!done) {
    // the single launch may have counted some levels before it stopped
    GB_CK(cudaMemsetAsync(eptr, 0, sizeof(int64_t) * (t->nleaf + 1), s));
    GB_CK(cudaMemsetAsync(d_pairs, 0, sizeof(unsigned long long), s));
    int64_t nf = 1;
    int64_t* d_seg = alloc_n<int64_t>(a, 3);
    int2* fr = alloc_n<int2>(a, 1);
    {
      int2 h = make_int2(0, 0);
      GB_CK(cudaMemcpyAsync(fr, &h, sizeof(int2), cudaMemcpyHostToDevice, s));
    }
    while (nf > 0) {
      const int64_t nb = blocks(nf);
      int64_t* cnt = alloc_n<int64_t>(a, 3 * nb);
      k_trav_count<<<(unsigned)nb, kThreads, 0, s>>>(fr, nf, cv, theta2, circ, cnt);
      GB_LAUNCH("k_trav_count");
      // one scan over the three segments of block totals; the segment starts
      // and the total are read back together (one host synchronisation per level)
      int64_t* scanned = cnt;
      scan_exclusive_i64_dev(a, scanned, 3 * nb, d_seg + 2, s);
      GB_CK(cudaMemcpyAsync(&d_seg[0], scanned + nb, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
      GB_CK(cudaMemcpyAsync(&d_seg[1], scanned + 2 * nb, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
      int64_t seg[3];
      GB_CK(cudaMemcpyAsync(seg, d_seg, sizeof(seg), cudaMemcpyDeviceToHost, s));
      host_sync(a, s);
      const int64_t total = seg[2];
      const int64_t n_next = seg[0], n_m = seg[1] - seg[0], n_p = total - seg[1];
      auto grow1 = [&](int32_t*& buf, int64_t nc, int64_t used) {
        int32_t* nb = alloc_n<int32_t>(a, nc);
        GB_CK(cudaMemcpyAsync(nb, buf, sizeof(int32_t) * used, cudaMemcpyDeviceToDevice, s));
        a.release(buf);
        buf = nb;
      };
      auto grow = [&](PairList& l, int64_t& cap, int64_t used, int64_t need) {
        if (used + need <= cap) return;
        const int64_t nc = std::max(2 * cap, used + need);
        grow1(l.tgt, nc, used);
        grow1(l.src, nc, used);
        cap = nc;
      };
      if (nm + n_m > cap_m) {
        const int64_t nc = std::max(2 * cap_m, nm + n_m);
        uint32_t* no = alloc_n<uint32_t>(a, nc);
        GB_CK(cudaMemcpyAsync(no, t->m2l_off, sizeof(uint32_t) * nm, cudaMemcpyDeviceToDevice, s));
        a.release(t->m2l_off);
        t->m2l_off = no;
      }
      grow(m2l, cap_m, nm, n_m);
      grow(p2p, cap_p, np, n_p);
      int2* next = alloc_n<int2>(a, n_next);
      k_trav_write<<<(unsigned)nb, kThreads, 0, s>>>(fr, nf, cv, theta2, circ, scanned, seg[0], seg[1], next, m2l,
                                                     nm, p2p, np, t->m2l_has, t->m2l_maxd, t->m2l_off);
      GB_LAUNCH("k_trav_write");
      nm += n_m;
      np += n_p;
      a.release(cnt);
      a.release(fr);
      fr = next;
      nf = n_next;
    }
    a.release(fr);
    a.release(d_seg);
    // the M2L cells and the largest class offset
    TravState* d_st = alloc_n<TravState>(a, 1);
    GB_CK(cudaMemsetAsync(d_st, 0, sizeof(TravState), s));
    k_count_flags<<<blocks(t->ncell), kThreads, 0, s>>>(t->m2l_has, t->ncell, d_st);
    GB_LAUNCH("k_count_flags");
    TravState h;
    GB_CK(cudaMemcpyAsync(&h, d_st, sizeof(TravState), cudaMemcpyDeviceToHost, s));
    GB_CK(cudaMemcpyAsync(&t->m2l_maxd_host, t->m2l_maxd, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    host_sync(a, s);
    t->m2l_ntgt = h.ntgt;
    a.release(d_st);
  }
  if (r2) a.release(r2);
  if (rr) a.release(rr);

  // The pairs stay in traversal order (deterministic: every offset comes from
  // an exclusive scan); only the inspection call sorts a copy by (target,
  // source).  Nothing on the evaluation path depends on that order.
  t->n_m2l = nm;
  t->n_p2p = np;
  t->m2l_tgt = m2l.tgt;
  t->m2l_src = m2l.src;
  t->p2p_tgt = p2p.tgt;
  t->p2p_src = p2p.src;

  // --- P2P body ranges per target leaf, merged where contiguous.  The
  // single-launch traversal counted each leaf's sources and the body pairs
  // already; the per-level one leaves it to k_p2p_leaf_count.
  if (!done) {
    k_p2p_leaf_count<<<blocks(np), kThreads, 0, s>>>(t->p2p_tgt, t->p2p_src, np, t->leaf_of_cell, t->c.bbeg,
                                                     t->c.bend, eptr, d_pairs);
    GB_LAUNCH("k_p2p_leaf_count");
  }
  scan_exclusive_i64(a, eptr, t->nleaf + 1, s);
  int32_t* cursor = alloc_n<int32_t>(a, t->nleaf);
  GB_CK(cudaMemsetAsync(cursor, 0, sizeof(int32_t) * t->nleaf, s));
  int32_t* rtmp = alloc_n<int32_t>(a, np);
  k_p2p_leaf_scatter<<<blocks(np), kThreads, 0, s>>>(t->p2p_tgt, t->p2p_src, np, t->leaf_of_cell, eptr, cursor,
                                                     rtmp);
  GB_LAUNCH("k_p2p_leaf_scatter");
  int32_t* rval = alloc_n<int32_t>(a, np);
  k_p2p_leaf_sort<<<(unsigned)((t->nleaf + kLeavesPerSortBlock - 1) / kLeavesPerSortBlock), 32 * kLeavesPerSortBlock, 0,
                    s>>>(eptr, (int)t->nleaf, t->c.bbeg, rtmp, rval);
  GB_LAUNCH("k_p2p_leaf_sort");
  a.release(cursor);
  a.release(rtmp);
  // per leaf: the number of merged ranges, then the ranges
  int64_t* rcount = alloc_n<int64_t>(a, t->nleaf + 1);
  GB_CK(cudaMemsetAsync(rcount, 0, sizeof(int64_t) * (t->nleaf + 1), s));
  const unsigned mblocks = (unsigned)((t->nleaf + kMergeWarps - 1) / kMergeWarps);
  k_merge_ranges<<<mblocks, 32 * kMergeWarps, 0, s>>>(eptr, rval, t->c.bbeg, t->c.bend, t->nleaf, rcount,
                                                      nullptr, nullptr);
  GB_LAUNCH("k_merge_ranges");
  // a leaf's merged ranges are at most its source leaves: np entries suffice
  scan_exclusive_i64_dev(a, rcount, t->nleaf + 1, reinterpret_cast<int64_t*>(t->d_tail), s);
  t->p2p_ranges = alloc_n<int2>(a, np);
  k_merge_ranges<<<mblocks, 32 * kMergeWarps, 0, s>>>(eptr, rval, t->c.bbeg, t->c.bend, t->nleaf, nullptr,
                                                      rcount, t->p2p_ranges);
  GB_LAUNCH("k_merge_ranges");
  t->p2p_rptr = alloc_n<int32_t>(a, t->nleaf + 1);
  k_i64_to_i32<<<blocks(t->nleaf + 1), kThreads, 0, s>>>(rcount, t->nleaf + 1, t->p2p_rptr);
  GB_LAUNCH("k_i64_to_i32");
  a.release(rval);
  a.release(eptr);
  a.release(rcount);
  if (t->flags & FMM_FLAG_MUTUAL_P2P) {
    int64_t* off = alloc_n<int64_t>(a, np);
    k_upair_flags<<<blocks(np), kThreads, 0, s>>>(t->p2p_tgt, t->p2p_src, np, off);
    GB_LAUNCH("k_upair_flags");
    t->n_p2p_upairs = scan_exclusive_i64_total(a, off, np, s);
    t->p2p_upairs = alloc_n<int2>(a, t->n_p2p_upairs);
    k_upair_write<<<blocks(np), kThreads, 0, s>>>(t->p2p_tgt, t->p2p_src, np, off, t->p2p_upairs);
    GB_LAUNCH("k_upair_write");
    a.release(off);
  }
}

}  // namespace gbfmm
