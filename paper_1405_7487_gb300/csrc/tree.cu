// tree.cu -- bounding cube, Morton keys, sort and level-wise octree
// construction (Sec. II.B: three key bits per level, 21 levels in 64 bits;
// Sec. II.C: a local tree built from the local bounding box; Sec. III.A:
// N_crit is the maximum number of bodies per leaf).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "common.cuh"
#include "grid.cuh"

namespace gbfmm {
namespace {

constexpr int kThreads = 256;

template <class R>
struct Body4;
template <>
struct Body4<float> {
  using type = float4;
};
template <>
struct Body4<double> {
  using type = double4_32a;
};

// Block-wide min of r[0..2] and max of r[3..6], into thread 0's r.
template <class R>
__device__ __forceinline__ void block_minmax7(R r[7]) {
  for (int o = 16; o > 0; o >>= 1)
    for (int k = 0; k < 7; ++k) {
      const R v = __shfl_down_sync(0xffffffffu, r[k], o);
      r[k] = k < 3 ? fmin(r[k], v) : fmax(r[k], v);
    }
  __shared__ R sh[kThreads / 32][7];
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
    for (int k = 0; k < 7; ++k) sh[w][k] = r[k];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int ww = 1; ww < (int)(blockDim.x >> 5); ++ww)
      for (int k = 0; k < 7; ++k) r[k] = k < 3 ? fmin(r[k], sh[ww][k]) : fmax(r[k], sh[ww][k]);
}

// Per-block min/max of each axis and a non-finite flag.  Minima and maxima
// are exact in the input's own precision, so the single-precision path
// reduces in FP32 (no FP64 per body) and widens each thread's result.
template <class R>
__global__ void k_bbox_partial(const R* __restrict__ xyzq, int64_t n, double* __restrict__ part) {
  // r: min x, y, z, max x, y, z, non-finite flag
  R r[7] = {(R)INFINITY, (R)INFINITY, (R)INFINITY, -(R)INFINITY, -(R)INFINITY, -(R)INFINITY, (R)0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const R x = xyzq[4 * i], y = xyzq[4 * i + 1], z = xyzq[4 * i + 2], q = xyzq[4 * i + 3];
    if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(q))) {
      r[6] = (R)1;
      continue;
    }
    r[0] = fmin(r[0], x); r[3] = fmax(r[3], x);
    r[1] = fmin(r[1], y); r[4] = fmax(r[4], y);
    r[2] = fmin(r[2], z); r[5] = fmax(r[5], z);
  }
  block_minmax7(r);
  if (threadIdx.x == 0)
    for (int k = 0; k < 7; ++k) part[7 * blockIdx.x + k] = (double)r[k];  // exact
}

// Root cube: centre (lo+hi)/2, half side H = max_axis (hi-lo)/2 * (1 + 2^-20)
// (H = 0.5 if all bodies coincide), corner = centre - H.  Explicitly rounded
// double operations: no fused multiply-add may change the keys.  The
// partials hold values of the input's precision R, so they are reduced in R.
template <class R>
__global__ void k_bbox_final(const double* __restrict__ part, int nb, double* __restrict__ root,
                             int* __restrict__ nonfinite) {
  // min/max are exact, so the reduction order does not matter
  R rr[7] = {(R)INFINITY, (R)INFINITY, (R)INFINITY, -(R)INFINITY, -(R)INFINITY, -(R)INFINITY, (R)0};
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    for (int a = 0; a < 3; ++a) {
      rr[a] = fmin(rr[a], (R)part[7 * b + a]);
      rr[3 + a] = fmax(rr[3 + a], (R)part[7 * b + 3 + a]);
    }
    rr[6] = fmax(rr[6], (R)part[7 * b + 6]);
  }
  block_minmax7(rr);
  if (threadIdx.x != 0) return;
  double r[7];
  for (int k = 0; k < 7; ++k) r[k] = (double)rr[k];
  *nonfinite = r[6] != 0.0;
  double h = 0.0;
  for (int a = 0; a < 3; ++a) {
    root[a] = r[a];
    root[3 + a] = r[3 + a];
    root[6 + a] = __dmul_rn(__dadd_rn(r[a], r[3 + a]), 0.5);
    h = fmax(h, __dmul_rn(__dsub_rn(r[3 + a], r[a]), 0.5));
  }
  double H = __dmul_rn(h, 1.0 + 0x1p-20);
  if (H == 0.0) H = 0.5;
  root[9] = H;
  for (int a = 0; a < 3; ++a) root[10 + a] = __dsub_rn(root[6 + a], H);
}

__device__ __forceinline__ uint64_t spread_bits(uint64_t v) {
  v &= 0x1fffffull;
  v = (v | (v << 32)) & 0x1f00000000ffffull;
  v = (v | (v << 16)) & 0x1f0000ff0000ffull;
  v = (v | (v << 8)) & 0x100f00f00f00f00full;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}

// Integer coordinate k = min(floor((x - corner) * S), 2^21 - 1) per axis,
// S = 2^21 / (2H) rounded once, interleaved x-major into a 63-bit key; idx
// (the identity permutation the sort starts from) is written when it is not
// null.  Each operation is an explicitly rounded double operation, as in the
// oracle, so the keys agree bit for bit.
template <class R>
__global__ void k_keys(const R* __restrict__ xyzq, int64_t n, const double* __restrict__ root,
                       uint64_t* __restrict__ keys, int32_t* __restrict__ idx) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double S = __ddiv_rn(2097152.0, __dadd_rn(root[9], root[9]));
  uint64_t key = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double d = __dsub_rn((double)xyzq[4 * i + a], root[10 + a]);
    double f = floor(__dmul_rn(d, S));
    int64_t k = (int64_t)f;
    k = k < 0 ? 0 : (k > 2097151 ? 2097151 : k);
    key |= spread_bits((uint64_t)k) << (2 - a);
  }
  keys[i] = key;
  if (idx) idx[i] = (int32_t)i;
}

template <class R>
__global__ void k_gather_bodies(const R* __restrict__ xyzq, const int32_t* __restrict__ perm,
                                int64_t n, typename Body4<R>::type* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t j = perm[i];
  typename Body4<R>::type b;
  b.x = xyzq[4 * j];
  b.y = xyzq[4 * j + 1];
  b.z = xyzq[4 * j + 2];
  b.w = xyzq[4 * j + 3];
  out[i] = b;
}

// First position in [s, e) whose octant digit (at the given shift) is >= d.
__device__ __forceinline__ int lower_digit(const uint64_t* __restrict__ keys, int s, int e, int shift,
                                           int d) {
  int lo = s, hi = e;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if ((int)((keys[mid] >> shift) & 7ull) < d) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Children of the cells of one level: a cell with more than ncrit bodies
// (and below level 21) splits into its nonempty octants, in Morton order.
// Eight lanes per cell: lane d finds where octant d starts (one binary
// search over the cell's sorted keys), its neighbour's start is its end, and
// a ballot over the eight lanes numbers the nonempty octants.
struct Octants {
  int c, d, s, e, b, nb;
  bool valid, split;
  unsigned group;  // nonempty-octant bits of this cell's eight lanes
};

// Lanes d = 0..7 of an aligned group of eight lanes take octant d of cell
// `cell` (valid false: no cell).  The cell arrays are read through L2: the
// cooperative level kernel reads cells that other blocks wrote.
// bnd: where octant d starts, per cell (8 entries a cell, relative to the
// level's first cell lb): the count pass writes it (saved = false), the write
// pass reads it back instead of searching again (saved = true).
__device__ __forceinline__ Octants octants_at(const uint64_t* __restrict__ keys, const int32_t* bbeg,
                                              const int32_t* bend, int cell, int d, bool valid, int level,
                                              int ncrit, int* bnd, int lb, bool saved) {
  Octants o;
  o.c = cell;
  o.d = d;
  o.valid = valid;
  o.s = valid ? __ldcg(bbeg + cell) : 0;
  o.e = valid ? __ldcg(bend + cell) : 0;
  o.split = valid && o.e - o.s > ncrit && level < kMaxLevel;
  o.b = o.s;
  if (o.split && d > 0) {
    int* at = bnd + 8 * (int64_t)(cell - lb) + d;
    if (saved) {
      o.b = *at;
    } else {
      o.b = lower_digit(keys, o.s, o.e, 3 * (kMaxLevel - level - 1), d);
      *at = o.b;
    }
  }
  o.nb = __shfl_down_sync(0xffffffffu, o.b, 1, 8);
  if (d == 7) o.nb = o.e;
  const unsigned m = __ballot_sync(0xffffffffu, o.split && o.nb > o.b);
  o.group = (m >> (threadIdx.x & 24)) & 0xffu;
  return o;
}

inline unsigned blocks(int64_t n, int t = kThreads) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------- levels
// All levels and the leaf list in one cooperative launch (every block is
// resident, so blocks can wait for one another).  Level l's cells are split
// into contiguous chunks, one per block; a level takes two grid barriers:
//   count: each block counts the children of its cells (eight lanes per cell,
//          as in octants_at()) and publishes its total;
//   write: each block adds the totals of the blocks before it (the children
//          of a level keep their parents' order, so the cell order is the
//          breadth-first (level, Morton) order) and writes its children.
// The barrier waits are bounded; one that runs out sets kErrGrid and an abort
// flag that ends every other wait.
struct LevelState {
  int level_begin[kMaxLevel + 3];  // first cell of each level, then the end
  int nlevel, ncell, nleaf, overflow;
  GridBar bar;
};

__global__ void __launch_bounds__(kThreads) k_tree_levels(const uint64_t* __restrict__ keys, int n, int ncrit,
                                                          int cap, Cells c, int32_t* __restrict__ leaves,
                                                          int32_t* __restrict__ leaf_of, int* __restrict__ partial,
                                                          int* __restrict__ bnd, LevelState* __restrict__ st,
                                                          int* __restrict__ err) {
  __shared__ int pass_cnt[kThreads / 8];
  __shared__ int chunk_sum;
  const int G = gridDim.x, blk = blockIdx.x;
  const int lane8 = threadIdx.x & 7, slot = threadIdx.x >> 3;  // 32 cells per pass
  if (blk == 0 && threadIdx.x == 0) {
    c.level[0] = 0;
    c.bbeg[0] = 0;
    c.bend[0] = n;
    c.ix[0] = c.iy[0] = c.iz[0] = 0;
    c.parent[0] = -1;
  }
  int lb = 0, le = 1, nlevel = 0;
  bool fine = grid_barrier(&st->bar, err), over = false;
  for (int l = 0; fine && le > lb; ++l) {
    nlevel = l + 1;
    const int ncur = le - lb, ch = (ncur + G - 1) / G;
    const int c0 = lb + min(blk * ch, ncur), c1 = lb + min((blk + 1) * ch, ncur);
    // count
    if (threadIdx.x == 0) chunk_sum = 0;
    __syncthreads();
    for (int cb = c0; cb < c1; cb += kThreads / 8) {
      const int cell = cb + slot;
      const Octants o = octants_at(keys, c.bbeg, c.bend, cell, lane8, cell < c1, l, ncrit, bnd, lb, false);
      if (o.valid && lane8 == 0) atomicAdd(&chunk_sum, __popc(o.group));
    }
    __syncthreads();
    if (threadIdx.x == 0) partial[blk] = chunk_sum;
    fine = grid_barrier(&st->bar, err);
    if (!fine) break;
    int before, total;
    block_prefix_totals<int, 1>(partial, blk, G, &before, &total);
    if ((int64_t)le + total > cap) {  // every block sees the same total
      if (blk == 0 && threadIdx.x == 0) st->overflow = 1;
      over = true;
      break;
    }
    // write
    int run = le + before;
    for (int cb = c0; cb < c1; cb += kThreads / 8) {
      const int cell = cb + slot;
      const Octants o = octants_at(keys, c.bbeg, c.bend, cell, lane8, cell < c1, l, ncrit, bnd, lb, true);
      const int nchild = __popc(o.group);
      if (lane8 == 0) pass_cnt[slot] = o.valid ? nchild : 0;
      __syncthreads();
      int k0 = run;
      for (int q = 0; q < slot; ++q) k0 += pass_cnt[q];
      int pass_total = 0;
      for (int q = 0; q < kThreads / 8; ++q) pass_total += pass_cnt[q];
      if (o.valid) {
        if ((o.group >> lane8) & 1u) {
          const int k = k0 + __popc(o.group & ((1u << lane8) - 1u));
          c.bbeg[k] = o.b;
          c.bend[k] = o.nb;
          c.ix[k] = 2 * __ldcg(c.ix + cell) + ((lane8 >> 2) & 1);
          c.iy[k] = 2 * __ldcg(c.iy + cell) + ((lane8 >> 1) & 1);
          c.iz[k] = 2 * __ldcg(c.iz + cell) + (lane8 & 1);
          c.parent[k] = cell;
          c.level[k] = l + 1;
        }
        if (lane8 == 0) {
          c.cbeg[cell] = nchild > 0 ? k0 : -1;
          c.nch[cell] = nchild;
        }
      }
      run += pass_total;
      __syncthreads();
    }
    if (blk == 0 && threadIdx.x == 0) st->level_begin[l + 1] = le;
    lb = le;
    le += total;
    fine = grid_barrier(&st->bar, err);
  }
  if (!fine || over) return;
  const int ncell = le;
  // leaves, in cell order
  {
    const int ch = (ncell + G - 1) / G;
    const int c0 = min(blk * ch, ncell), c1 = min((blk + 1) * ch, ncell);
    if (threadIdx.x == 0) chunk_sum = 0;
    __syncthreads();
    for (int i = c0 + threadIdx.x; i < c1; i += blockDim.x)
      if (__ldcg(c.nch + i) == 0) atomicAdd(&chunk_sum, 1);
    __syncthreads();
    if (threadIdx.x == 0) partial[blk] = chunk_sum;
    if (!grid_barrier(&st->bar, err)) return;
    int before, total;
    block_prefix_totals<int, 1>(partial, blk, G, &before, &total);
    __shared__ int wcnt[kThreads / 32];
    int run = before;
    for (int cb = c0; cb < c1; cb += blockDim.x) {
      const int i = cb + threadIdx.x;
      const bool leaf = i < c1 && __ldcg(c.nch + i) == 0;
      const unsigned m = __ballot_sync(0xffffffffu, leaf);
      if ((threadIdx.x & 31) == 0) wcnt[threadIdx.x >> 5] = __popc(m);
      __syncthreads();
      int k = run + __popc(m & ((1u << (threadIdx.x & 31)) - 1u));
      int pass_total = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        if (w < (int)(threadIdx.x >> 5)) k += wcnt[w];
        pass_total += wcnt[w];
      }
      if (i < c1) {
        leaf_of[i] = leaf ? k : -1;
        if (leaf) leaves[k] = i;
      }
      run += pass_total;
      __syncthreads();
    }
    if (blk == 0 && threadIdx.x == 0) {
      st->level_begin[0] = 0;
      st->level_begin[nlevel] = ncell;
      st->nlevel = nlevel;
      st->ncell = ncell;
      st->nleaf = total;
    }
  }
}

template <class R>
void build_tree_impl(fmm_tree* t, const R* xyzq) {
  Arena& a = t->arena;
  cudaStream_t s = t->stream;
  const int64_t N = t->N;
  // --- bounding cube
  const int nb = (int)std::min<int64_t>(1024, (N + kThreads - 1) / kThreads);
  double* part = alloc_n<double>(a, 7 * (size_t)nb);
  t->d_root = alloc_n<double>(a, 13);
  int* d_bad = alloc_n<int>(a, 1);
  k_bbox_partial<R><<<nb, kThreads, 0, s>>>(xyzq, N, part);
  GB_LAUNCH("k_bbox_partial");
  k_bbox_final<R><<<1, kThreads, 0, s>>>(part, nb, t->d_root, d_bad);
  GB_LAUNCH("k_bbox_final");
  // --- keys and stable sort (ties keep input order: LSD radix is stable and
  // the initial order is the input order).  The root cube stays on the
  // device until the levels are read back; a non-finite input still gives
  // in-range keys (the conversion of NaN gives 0 and the key is clamped).
  uint64_t* keys = alloc_n<uint64_t>(a, N);
  int32_t* idx = alloc_n<int32_t>(a, N);
  k_keys<R><<<blocks(N), kThreads, 0, s>>>(xyzq, N, t->d_root, keys, idx);
  GB_LAUNCH("k_keys");
  radix_sort_pairs(a, keys, idx, N, 63, s);
  t->keys = keys;
  t->perm = idx;
  using B4 = typename Body4<R>::type;
  B4* bodies = alloc_n<B4>(a, N);
  k_gather_bodies<R><<<blocks(N), kThreads, 0, s>>>(xyzq, t->perm, N, bodies);
  GB_LAUNCH("k_gather_bodies");
  t->bodies = bodies;
  t->work = alloc_n<B4>(a, N);
  GB_CK(cudaMemcpyAsync(t->work, bodies, sizeof(B4) * N, cudaMemcpyDeviceToDevice, s));

  // --- levels and leaves: one cooperative launch, then one read-back of the
  // level sizes together with the root cube.  The cell arrays are sized for
  // 8 N / ncrit + 4096 cells first (the trees here hold 2 to 4 N / ncrit);
  // if the tree needs more, the launch is repeated at the bound
  // sum_l min(8^l, N, 8 floor(N / (ncrit + 1))), l <= 21.
  int sms = 0, dev = 0, per_sm = 0;
  GB_CK(cudaGetDevice(&dev));
  GB_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  GB_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tree_levels, kThreads, 0));
  const int G = std::max(1, std::min(4, per_sm) * sms);
  int64_t bound = 0;
  {
    const int64_t split_max = 8 * (N / ((int64_t)t->ncrit + 1));
    int64_t p8 = 1;
    for (int l = 0; l <= kMaxLevel; ++l) {
      bound += l == 0 ? 1 : std::min(std::min(p8, N), split_max);
      p8 = std::min<int64_t>(p8 * 8, 1ll << 40);
    }
  }
  if (bound > 0x7fffffff) bound = 0x7fffffff;
  int64_t cap = std::min<int64_t>(bound, 8 * ((N + t->ncrit - 1) / t->ncrit) + 4096);
  // GBFMM_TREE_CELLS overrides the first capacity (the test of the retry)
  if (const char* env = getenv("GBFMM_TREE_CELLS")) cap = std::min<int64_t>(bound, std::max<int64_t>(1, atoll(env)));
  int* partial = alloc_n<int>(a, G);
  LevelState* d_st = alloc_n<LevelState>(a, 1);
  int* bnd = nullptr;  // octant starts of one level's cells (at most cap cells)
  LevelState hst;
  double hroot[13];
  int hbad = 0;
  for (int attempt = 0;; ++attempt) {
    Cells& c = t->c;
    int32_t** fields[9] = {&c.level, &c.ix, &c.iy, &c.iz, &c.bbeg, &c.bend, &c.cbeg, &c.nch, &c.parent};
    for (auto f : fields) *f = alloc_n<int32_t>(a, cap);
    t->leaves = alloc_n<int32_t>(a, cap);
    t->leaf_of_cell = alloc_n<int32_t>(a, cap);
    bnd = alloc_n<int>(a, 8 * (size_t)cap);
    GB_CK(cudaMemsetAsync(d_st, 0, sizeof(LevelState), s));
    const int n32 = (int)N, ncrit = t->ncrit, cap32 = (int)cap;
    int* err = a.err;
    void* args[] = {(void*)&keys, (void*)&n32, (void*)&ncrit, (void*)&cap32, (void*)&c,
                    (void*)&t->leaves, (void*)&t->leaf_of_cell, (void*)&partial, (void*)&bnd, (void*)&d_st,
                    (void*)&err};
    GB_CK(cudaLaunchCooperativeKernel((const void*)k_tree_levels, dim3(G), dim3(kThreads), args, 0, s));
    GB_LAUNCH("k_tree_levels");
    GB_CK(cudaMemcpyAsync(&hst, d_st, sizeof(LevelState), cudaMemcpyDeviceToHost, s));
    if (attempt == 0) {
      GB_CK(cudaMemcpyAsync(hroot, t->d_root, sizeof(hroot), cudaMemcpyDeviceToHost, s));
      GB_CK(cudaMemcpyAsync(&hbad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    check_scan_error(a, s);  // synchronises; a grid wait past its limit is FMM_ERR_TIMEOUT
    if (attempt == 0 && hbad) fail(FMM_ERR_NONFINITE, "non-finite position or charge");
    if (!hst.overflow) break;
    if (cap >= bound) fail(FMM_ERR_ARG, "too many cells");
    for (auto f : fields) a.release(*f);
    a.release(t->leaves);
    a.release(t->leaf_of_cell);
    a.release(bnd);
    cap = bound;
  }
  a.release(bnd);
  a.release(partial);
  a.release(d_st);
  a.release(part);
  a.release(d_bad);
  for (int k = 0; k < 3; ++k) {
    t->root.lo[k] = hroot[k];
    t->root.hi[k] = hroot[3 + k];
    t->root.centre[k] = hroot[6 + k];
    t->root.corner[k] = hroot[10 + k];
  }
  t->root.H = hroot[9];
  t->nlevel = hst.nlevel;
  t->ncell = hst.ncell;
  t->nleaf = hst.nleaf;
  t->level_begin.assign(hst.level_begin, hst.level_begin + hst.nlevel + 1);
}

}  // namespace

void build_tree(fmm_tree* t, const void* xyzq, bool f64) {
  if (f64) build_tree_impl<double>(t, static_cast<const double*>(xyzq));
  else build_tree_impl<float>(t, static_cast<const float*>(xyzq));
}

}  // namespace gbfmm

// ---------------------------------------------------------------------------
// Allocation-free root cube and Morton keys.
//
// The paper has no counterpart of this entry point.  It serves callers that
// may not allocate device memory while they call this library: code running
// under a fixed device-memory budget or inside another framework's allocator
// (which owns every allocation), and code that must not trigger the device-
// wide synchronisation a cudaMalloc/cudaFree can cause in the middle of its
// own stream work.  It is the first step of fmm_build (bounding cube and
// keys) with the reduction's scratch held in a fixed file-scope device array
// instead of workspace from an allocator.
namespace gbfmm {
namespace {

constexpr int kNoAllocBlocks = 1024;  // partial boxes of at most 1024 blocks
constexpr int kNoAllocBodies = 0x7fffffff;

// Partial bounding boxes (7 doubles per block) and the non-finite flag used
// when the caller passes none.  One copy per device, kept until exit
// (about 57 KB); every call overwrites it.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocBlocks * 7 + 32];

// The scratch array's device address per CUDA context (the address belongs
// to the context the module was loaded in).  The runtime uses the primary
// context of the current device unless the caller made another current.
std::mutex g_noalloc_mu;
std::vector<std::pair<CUcontext, double*>> g_noalloc_ptr;

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);

// cuCtxGetCurrent from the driver, found through the runtime (the library
// does not link libcuda); null if unavailable
CUcontext current_context() {
  static CtxGetCurrentFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    return reinterpret_cast<CtxGetCurrentFn>(p);
  }();
  CUcontext c = nullptr;
  if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

}  // namespace
}  // namespace gbfmm

extern "C" int fmm_root_keys_noalloc(const float* xyzq, int64_t n, double* root, uint64_t* keys,
                                     int32_t* nonfinite, fmm_stream stream) {
  using namespace gbfmm;
  if (!xyzq || !root || n < 1) return FMM_ERR_ARG;
  if (n > kNoAllocBodies) {
    g_last_error = "fmm_root_keys_noalloc: n exceeds the maximum of 2^31 - 1 bodies";
    return FMM_ERR_ARG;
  }
  double* scratch = nullptr;
  {
    // once per device (per CUDA context), with that device current: the
    // device address of the scratch array (the host-side symbol is only a
    // stand-in for it).  The lookup also makes the context current if the
    // runtime had not yet done so.
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    CUcontext ctx = current_context();
    for (auto& e : g_noalloc_ptr)
      if (ctx && e.first == ctx) scratch = e.second;
    if (!scratch) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        g_last_error = "fmm_root_keys_noalloc: cudaGetSymbolAddress failed";
        return FMM_ERR_CUDA;
      }
      scratch = static_cast<double*>(p);
      ctx = current_context();
      if (ctx) g_noalloc_ptr.emplace_back(ctx, scratch);
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int nb = (int)std::min<int64_t>(kNoAllocBlocks, (n + kThreads - 1) / kThreads);
  int* flag = nonfinite ? nonfinite : reinterpret_cast<int*>(scratch + kNoAllocBlocks * 7);
  k_bbox_partial<float><<<nb, kThreads, 0, s>>>(xyzq, n, scratch);
  k_bbox_final<float><<<1, kThreads, 0, s>>>(scratch, nb, root, flag);
  if (keys) k_keys<float><<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, s>>>(xyzq, n, root, keys, nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_last_error = std::string("fmm_root_keys_noalloc: ") + cudaGetErrorName(e);
    return FMM_ERR_CUDA;
  }
  return FMM_OK;
}
