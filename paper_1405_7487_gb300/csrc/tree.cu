// tree.cu -- bounding cube, Morton keys, sort and level-wise octree
// construction (Sec. II.B: three key bits per level, 21 levels in 64 bits;
// Sec. II.C: a local tree built from the local bounding box; Sec. III.A:
// N_crit is the maximum number of bodies per leaf).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "common.cuh"

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

// Per-block min/max of each axis and a non-finite flag.  Minima and maxima
// are exact in the input's own precision, so the single-precision path
// reduces in FP32 (no FP64 per body) and widens each thread's result.
template <class R>
__global__ void k_bbox_partial(const R* __restrict__ xyzq, int64_t n, double* __restrict__ part) {
  R lr[3] = {(R)INFINITY, (R)INFINITY, (R)INFINITY}, hr[3] = {-(R)INFINITY, -(R)INFINITY, -(R)INFINITY};
  bool bad_r = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const R x = xyzq[4 * i], y = xyzq[4 * i + 1], z = xyzq[4 * i + 2], q = xyzq[4 * i + 3];
    if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(q))) {
      bad_r = true;
      continue;
    }
    lr[0] = fmin(lr[0], x); hr[0] = fmax(hr[0], x);
    lr[1] = fmin(lr[1], y); hr[1] = fmax(hr[1], y);
    lr[2] = fmin(lr[2], z); hr[2] = fmax(hr[2], z);
  }
  double lo[3], hi[3], bad = bad_r ? 1.0 : 0.0;
  for (int a = 0; a < 3; ++a) {
    lo[a] = (double)lr[a];
    hi[a] = (double)hr[a];
  }
  for (int o = 16; o > 0; o >>= 1) {
    for (int a = 0; a < 3; ++a) {
      lo[a] = fmin(lo[a], __shfl_down_sync(0xffffffffu, lo[a], o));
      hi[a] = fmax(hi[a], __shfl_down_sync(0xffffffffu, hi[a], o));
    }
    bad = fmax(bad, __shfl_down_sync(0xffffffffu, bad, o));
  }
  __shared__ double s[kThreads / 32][7];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    for (int a = 0; a < 3; ++a) {
      s[w][a] = lo[a];
      s[w][3 + a] = hi[a];
    }
    s[w][6] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double r[7];
    for (int k = 0; k < 7; ++k) r[k] = s[0][k];
    for (int ww = 1; ww < kThreads / 32; ++ww) {
      for (int a = 0; a < 3; ++a) {
        r[a] = fmin(r[a], s[ww][a]);
        r[3 + a] = fmax(r[3 + a], s[ww][3 + a]);
      }
      r[6] = fmax(r[6], s[ww][6]);
    }
    for (int k = 0; k < 7; ++k) part[7 * blockIdx.x + k] = r[k];
  }
}

// Root cube: centre (lo+hi)/2, half side H = max_axis (hi-lo)/2 * (1 + 2^-20)
// (H = 0.5 if all bodies coincide), corner = centre - H.  Explicitly rounded
// double operations: no fused multiply-add may change the keys.
__global__ void k_bbox_final(const double* __restrict__ part, int nb, double* __restrict__ root,
                             int* __restrict__ nonfinite) {
  // min/max are exact, so the reduction order does not matter
  __shared__ double sh[kThreads / 32][7];
  double r[7] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY, 0.0};
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    for (int a = 0; a < 3; ++a) {
      r[a] = fmin(r[a], part[7 * b + a]);
      r[3 + a] = fmax(r[3 + a], part[7 * b + 3 + a]);
    }
    r[6] = fmax(r[6], part[7 * b + 6]);
  }
  for (int o = 16; o > 0; o >>= 1)
    for (int k = 0; k < 7; ++k) {
      const double v = __shfl_down_sync(0xffffffffu, r[k], o);
      r[k] = k < 3 ? fmin(r[k], v) : fmax(r[k], v);
    }
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
    for (int k = 0; k < 7; ++k) sh[warp][k] = r[k];
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
    for (int a = 0; a < 3; ++a) {
      r[a] = fmin(r[a], sh[w][a]);
      r[3 + a] = fmax(r[3 + a], sh[w][3 + a]);
    }
    r[6] = fmax(r[6], sh[w][6]);
  }
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

// Integer coordinate k = min(floor((x - corner) / (2H) * 2^21), 2^21 - 1) per
// axis, interleaved x-major into a 63-bit key; idx (the identity permutation
// the sort starts from) is written when it is not null.
template <class R>
__global__ void k_keys(const R* __restrict__ xyzq, int64_t n, const double* __restrict__ root,
                       uint64_t* __restrict__ keys, int32_t* __restrict__ idx) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double side = __dadd_rn(root[9], root[9]);
  uint64_t key = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double d = __dsub_rn((double)xyzq[4 * i + a], root[10 + a]);
    double s = __dmul_rn(__ddiv_rn(d, side), 2097152.0);
    double f = floor(s);
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

__device__ __forceinline__ Octants octants(const uint64_t* __restrict__ keys, const int32_t* __restrict__ bbeg,
                                           const int32_t* __restrict__ bend, int ncell, int level, int ncrit) {
  Octants o;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  o.c = g >> 3;
  o.d = g & 7;
  o.valid = o.c < ncell;
  o.s = o.valid ? bbeg[o.c] : 0;
  o.e = o.valid ? bend[o.c] : 0;
  o.split = o.valid && o.e - o.s > ncrit && level < kMaxLevel;
  o.b = o.s;
  if (o.split && o.d > 0) o.b = lower_digit(keys, o.s, o.e, 3 * (kMaxLevel - level - 1), o.d);
  o.nb = __shfl_down_sync(0xffffffffu, o.b, 1, 8);
  if (o.d == 7) o.nb = o.e;
  const unsigned m = __ballot_sync(0xffffffffu, o.split && o.nb > o.b);
  o.group = (m >> (threadIdx.x & 24)) & 0xffu;
  return o;
}

__global__ void k_split_count(const uint64_t* __restrict__ keys, const int32_t* __restrict__ bbeg,
                              const int32_t* __restrict__ bend, int ncell, int level, int ncrit,
                              int64_t* __restrict__ nchild) {
  const Octants o = octants(keys, bbeg, bend, ncell, level, ncrit);
  if (o.valid && o.d == 0) nchild[o.c] = __popc(o.group);
}

__global__ void k_split_write(const uint64_t* __restrict__ keys, const int32_t* __restrict__ bbeg,
                              const int32_t* __restrict__ bend, const int32_t* __restrict__ ix,
                              const int32_t* __restrict__ iy, const int32_t* __restrict__ iz,
                              int ncell, int level, int ncrit, int first_cell, int first_child,
                              const int64_t* __restrict__ off, int32_t* __restrict__ cbeg,
                              int32_t* __restrict__ nch, int32_t* __restrict__ o_bbeg,
                              int32_t* __restrict__ o_bend, int32_t* __restrict__ o_ix,
                              int32_t* __restrict__ o_iy, int32_t* __restrict__ o_iz,
                              int32_t* __restrict__ o_parent) {
  const Octants o = octants(keys, bbeg, bend, ncell, level, ncrit);
  if (!o.valid) return;
  const int k0 = (int)off[o.c];
  const int n = __popc(o.group);
  if ((o.group >> o.d) & 1u) {
    const int k = k0 + __popc(o.group & ((1u << o.d) - 1u));
    o_bbeg[k] = o.b;
    o_bend[k] = o.nb;
    o_ix[k] = 2 * ix[o.c] + ((o.d >> 2) & 1);
    o_iy[k] = 2 * iy[o.c] + ((o.d >> 1) & 1);
    o_iz[k] = 2 * iz[o.c] + (o.d & 1);
    o_parent[k] = first_cell + o.c;
  }
  if (o.d == 0) {
    cbeg[o.c] = n > 0 ? first_child + k0 : -1;
    nch[o.c] = n;
  }
}

__global__ void k_leaf_flags(const int32_t* __restrict__ nch, int n, int64_t* __restrict__ f) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) f[i] = nch[i] == 0;
}

__global__ void k_leaf_compact(const int32_t* __restrict__ nch, const int64_t* __restrict__ off,
                               int n, int32_t* __restrict__ leaves, int32_t* __restrict__ leaf_of) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (nch[i] == 0) {
    leaves[off[i]] = i;
    leaf_of[i] = (int32_t)off[i];
  } else {
    leaf_of[i] = -1;
  }
}

inline unsigned blocks(int64_t n, int t = kThreads) { return (unsigned)((n + t - 1) / t); }

// The root cell: all bodies, integer coordinates 0, no parent.
__global__ void k_root_cell(int32_t n, int32_t* bbeg, int32_t* bend, int32_t* ix, int32_t* iy, int32_t* iz,
                            int32_t* parent) {
  *bbeg = 0;
  *bend = n;
  *ix = *iy = *iz = 0;
  *parent = -1;
}

struct LevelArrays {
  int n = 0;
  int32_t *bbeg, *bend, *ix, *iy, *iz, *parent, *cbeg, *nch;
};

// One level's arrays for the concatenation kernel: its first cell and the
// eight per-cell fields (ix, iy, iz, bbeg, bend, cbeg, nch, parent).
struct LevelSrc {
  int first;
  const int32_t* f[8];
};

// Breadth-first cell arrays from the per-level arrays, every level in one
// launch: cell i finds its level by binary search over the first cells.
__global__ void k_concat_levels(const LevelSrc* __restrict__ lv, int nlevel, int ncell, int32_t* __restrict__ level,
                                int32_t* __restrict__ o0, int32_t* __restrict__ o1, int32_t* __restrict__ o2,
                                int32_t* __restrict__ o3, int32_t* __restrict__ o4, int32_t* __restrict__ o5,
                                int32_t* __restrict__ o6, int32_t* __restrict__ o7) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ncell) return;
  int lo = 0, hi = nlevel;  // last level whose first cell is <= i
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (lv[mid].first <= i) lo = mid;
    else hi = mid;
  }
  const LevelSrc& L = lv[lo];
  const int k = i - L.first;
  level[i] = lo;
  o0[i] = L.f[0][k];
  o1[i] = L.f[1][k];
  o2[i] = L.f[2][k];
  o3[i] = L.f[3][k];
  o4[i] = L.f[4][k];
  o5[i] = L.f[5][k];
  o6[i] = L.f[6][k];
  o7[i] = L.f[7][k];
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
  k_bbox_final<<<1, kThreads, 0, s>>>(part, nb, t->d_root, d_bad);
  GB_LAUNCH("k_bbox_final");
  double hroot[13];
  int hbad = 0;
  GB_CK(cudaMemcpyAsync(hroot, t->d_root, sizeof(hroot), cudaMemcpyDeviceToHost, s));
  GB_CK(cudaMemcpyAsync(&hbad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  host_sync(a, s);
  a.release(part);
  a.release(d_bad);
  if (hbad) fail(FMM_ERR_NONFINITE, "non-finite position or charge");
  for (int k = 0; k < 3; ++k) {
    t->root.lo[k] = hroot[k];
    t->root.hi[k] = hroot[3 + k];
    t->root.centre[k] = hroot[6 + k];
    t->root.corner[k] = hroot[10 + k];
  }
  t->root.H = hroot[9];
  // --- keys and stable sort (ties keep input order: LSD radix is stable and
  // the initial order is the input order)
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

  // --- levels
  std::vector<LevelArrays> lv;
  LevelArrays root;
  root.n = 1;
  root.bbeg = alloc_n<int32_t>(a, 1);
  root.bend = alloc_n<int32_t>(a, 1);
  root.ix = alloc_n<int32_t>(a, 1);
  root.iy = alloc_n<int32_t>(a, 1);
  root.iz = alloc_n<int32_t>(a, 1);
  root.parent = alloc_n<int32_t>(a, 1);
  k_root_cell<<<1, 1, 0, s>>>((int32_t)N, root.bbeg, root.bend, root.ix, root.iy, root.iz, root.parent);
  GB_LAUNCH("k_root_cell");
  lv.push_back(root);
  int first = 0;
  for (int l = 0;; ++l) {
    LevelArrays& cur = lv[l];
    cur.cbeg = alloc_n<int32_t>(a, cur.n);
    cur.nch = alloc_n<int32_t>(a, cur.n);
    int64_t* off = alloc_n<int64_t>(a, cur.n);
    k_split_count<<<blocks(8 * (int64_t)cur.n), kThreads, 0, s>>>(t->keys, cur.bbeg, cur.bend, cur.n, l,
                                                                   t->ncrit, off);
    GB_LAUNCH("k_split_count");
    const int64_t nnext = scan_exclusive_i64_total(a, off, cur.n, s);
    if (nnext > 0x7fffffff - first - cur.n) fail(FMM_ERR_ARG, "too many cells");
    LevelArrays nx;
    nx.n = (int)nnext;
    if (nnext > 0) {
      nx.bbeg = alloc_n<int32_t>(a, nnext);
      nx.bend = alloc_n<int32_t>(a, nnext);
      nx.ix = alloc_n<int32_t>(a, nnext);
      nx.iy = alloc_n<int32_t>(a, nnext);
      nx.iz = alloc_n<int32_t>(a, nnext);
      nx.parent = alloc_n<int32_t>(a, nnext);
    }
    k_split_write<<<blocks(8 * (int64_t)cur.n), kThreads, 0, s>>>(
        t->keys, cur.bbeg, cur.bend, cur.ix, cur.iy, cur.iz, cur.n, l, t->ncrit, first,
        first + cur.n, off, cur.cbeg, cur.nch, nx.bbeg, nx.bend, nx.ix, nx.iy, nx.iz, nx.parent);
    GB_LAUNCH("k_split_write");
    a.release(off);
    first += cur.n;
    if (nnext == 0) break;
    lv.push_back(nx);
  }
  // --- concatenate the levels (breadth-first cell order)
  t->nlevel = (int)lv.size();
  t->level_begin.assign(1, 0);
  for (auto& L : lv) t->level_begin.push_back(t->level_begin.back() + L.n);
  const int nc = t->level_begin.back();
  t->ncell = nc;
  Cells& c = t->c;
  int32_t** fields[9] = {&c.level, &c.ix, &c.iy, &c.iz, &c.bbeg, &c.bend, &c.cbeg, &c.nch, &c.parent};
  for (auto f : fields) *f = alloc_n<int32_t>(a, nc);
  {
    std::vector<LevelSrc> h(lv.size());
    for (size_t l = 0; l < lv.size(); ++l) {
      const LevelArrays& L = lv[l];
      h[l].first = t->level_begin[l];
      const int32_t* f[8] = {L.ix, L.iy, L.iz, L.bbeg, L.bend, L.cbeg, L.nch, L.parent};
      for (int k = 0; k < 8; ++k) h[l].f[k] = f[k];
    }
    LevelSrc* d = alloc_n<LevelSrc>(a, h.size());
    GB_CK(cudaMemcpyAsync(d, h.data(), sizeof(LevelSrc) * h.size(), cudaMemcpyHostToDevice, s));
    k_concat_levels<<<blocks(nc), kThreads, 0, s>>>(d, (int)h.size(), nc, c.level, c.ix, c.iy, c.iz, c.bbeg,
                                                     c.bend, c.cbeg, c.nch, c.parent);
    GB_LAUNCH("k_concat_levels");
    // the H2D copy reads h (pageable) before returning; d is freed in order
    a.release(d);
  }
  for (auto& L : lv) {
    int32_t* all[8] = {L.ix, L.iy, L.iz, L.bbeg, L.bend, L.cbeg, L.nch, L.parent};
    for (auto p : all) a.release(p);
  }
  // --- leaves
  int64_t* flag = alloc_n<int64_t>(a, nc);
  k_leaf_flags<<<blocks(nc), kThreads, 0, s>>>(c.nch, nc, flag);
  GB_LAUNCH("k_leaf_flags");
  t->nleaf = (int)scan_exclusive_i64_total(a, flag, nc, s);
  t->leaves = alloc_n<int32_t>(a, t->nleaf);
  t->leaf_of_cell = alloc_n<int32_t>(a, nc);
  k_leaf_compact<<<blocks(nc), kThreads, 0, s>>>(c.nch, flag, nc, t->leaves, t->leaf_of_cell);
  GB_LAUNCH("k_leaf_compact");
  a.release(flag);
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
  k_bbox_final<<<1, kThreads, 0, s>>>(scratch, nb, root, flag);
  if (keys) k_keys<float><<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, s>>>(xyzq, n, root, keys, nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_last_error = std::string("fmm_root_keys_noalloc: ") + cudaGetErrorName(e);
    return FMM_ERR_CUDA;
  }
  return FMM_OK;
}
