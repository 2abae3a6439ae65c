// ops.cu -- translation operators (set up in double precision) and the M2L
// plan: targets tiled kTile at a time, interactions grouped by translation
// operator.
//
// Expansions (Sec. II.A: P2M, M2M, M2L, L2L, L2P; the mathematics is that of
// the solid-harmonic FMM the paper cites):
//   Ups_n^m(r) = r^n P_n^m(cos t) e^{i m phi} / (n+m)!      (regular)
//   Th_n^m(r)  = (n-m)! P_n^m(cos t) e^{i m phi} / r^{n+1}   (irregular)
//   (Condon-Shortley phase, X_n^{-m} = (-1)^m conj(X_n^m)), so that
//   1/|x - y| = sum conj(Ups_n^m(y)) Th_n^m(x),
//   Ups(a + b) = sum Ups_k^l(a) Ups_{n-k}^{m-l}(b),
//   Th_n^m(x - y) = sum conj(Ups_k^l(y)) Th_{n+k}^{m+l}(x).
// Stored expansions are scaled by the cell half side R so that every
// operator depends only on the relative geometry:
//   M~_n^m = M_n^m / R_A^n,   L~_k^l = L_k^l R_B^{k+1}.
//   M2M  M~_n^m(P) = sum M~_k^l(C) 2^{-k} conj(Ups_{n-k}^{m-l}(t)),   t = (c_C - c_P)/R_P
//   L2L  L~_j^i(C) = sum L~_k^l(P) 2^{-(j+1)} conj(Ups_{k-j}^{l-i}(t))
//   M2L  L~_k^l(B) = (-1)^k sum M~_n^m(A) (R_B/r)^{k+1} (R_A/r)^n Th_{n+k}^{m+l}((c_B - c_A)/r),
//        r = min(R_A, R_B), so (c_B - c_A)/r is an integer vector.
// Each complex operator acts on the real packing of the m >= 0 coefficients
// (index n*n for Re X_n^0, n*n + 2m - 1 / n*n + 2m for Re / Im X_n^m) and is
// written out as a real Kp x Kp matrix.
#include <algorithm>
#include <cfloat>

#include "common.cuh"

namespace gbfmm {
namespace {

constexpr int kThreads = 256;
// Largest dense key table (log2 entries) of the M2L plan; beyond it the plan
// sorts the pairs instead.
constexpr int kDenseBits = 22;
inline unsigned blocks(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

struct cd {
  double re, im;
};
__device__ __forceinline__ cd cmul(cd a, cd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cd cconj(cd a) { return {a.re, -a.im}; }
__device__ __forceinline__ cd cscale(cd a, double s) { return {a.re * s, a.im * s}; }

__device__ __forceinline__ int tri(int n, int m) { return n * (n + 1) / 2 + m; }

// X_n^m for any -n <= m <= n from the m >= 0 triangle.
__device__ __forceinline__ cd hget(const cd* X, int n, int m) {
  if (m >= 0) return X[tri(n, m)];
  cd v = X[tri(n, -m)];
  v.im = -v.im;
  if ((-m) & 1) {
    v.re = -v.re;
    v.im = -v.im;
  }
  return v;
}

// Regular harmonics, degrees < P, into the m >= 0 triangle.  Thread m < P
// of the block forms column m: the diagonal term by m steps of
// Ups_m^m = -(x + i y) Ups_{m-1}^{m-1} / (2m), then the recurrence up the
// column.  Every entry takes the same operations as in a serial sweep of the
// triangle, so the values do not depend on the block size.
__device__ void regular_tri(double x, double y, double z, int P, cd* U) {
  const int m = threadIdx.x;
  if (m >= P) return;
  const double r2 = x * x + y * y + z * z;
  cd d{1.0, 0.0};
  for (int k = 1; k <= m; ++k) d = cscale(cmul(d, {-x, -y}), 1.0 / (2.0 * k));
  U[tri(m, m)] = d;
  for (int n = m + 1; n < P; ++n) {
    cd a = U[tri(n - 1, m)];
    cd b = n - 2 >= m ? U[tri(n - 2, m)] : cd{0.0, 0.0};
    double f = 1.0 / ((double)(n + m) * (double)(n - m));
    U[tri(n, m)] = {((2.0 * n - 1.0) * z * a.re - r2 * b.re) * f, ((2.0 * n - 1.0) * z * a.im - r2 * b.im) * f};
  }
}

// Irregular harmonics, degrees < P, into the m >= 0 triangle; thread m < P
// forms column m (as regular_tri).
__device__ void irregular_tri(double x, double y, double z, int P, cd* T) {
  const int m = threadIdx.x;
  if (m >= P) return;
  const double r2 = x * x + y * y + z * z;
  const double ir2 = 1.0 / r2;
  cd d{1.0 / sqrt(r2), 0.0};
  for (int k = 1; k <= m; ++k) d = cscale(cmul(d, {x, y}), -(2.0 * k - 1.0) * ir2);
  T[tri(m, m)] = d;
  for (int n = m + 1; n < P; ++n) {
    cd a = T[tri(n - 1, m)];
    cd b = n - 2 >= m ? T[tri(n - 2, m)] : cd{0.0, 0.0};
    double c1 = (2.0 * n - 1.0) * z, c2 = (double)(n + m - 1) * (double)(n - m - 1);
    T[tri(n, m)] = {(c1 * a.re - c2 * b.re) * ir2, (c1 * a.im - c2 * b.im) * ir2};
  }
}

__device__ __forceinline__ int ridx(int n, int m, int part) { return n * n + (m == 0 ? 0 : 2 * m - 1 + part); }

enum Kind { kM2M = 0, kL2L = 1, kM2L = 2 };

// Complex coefficient C(out (a, b), in (c, d)) for -c <= d <= c.
struct Coef {
  int kind;
  int eA, eB;  // M2L: R_A / r = 2^eA and R_B / r = 2^eB
  const cd* X;
  const double* scale;  // M2L: scale[a * kMaxP + c] = (-1)^a 2^(eB (a + 1) + eA c)
  __device__ cd operator()(int a, int b, int c, int d) const {
    if (kind == kM2L) {
      // out (k = a, l = b), in (n = c, m = d)
      return cscale(hget(X, a + c, d + b), scale[a * kMaxP + c]);
    }
    if (kind == kM2M) {
      // out (n = a, m = b), in (k = c, l = d)
      if (c > a) return {0.0, 0.0};
      int dm = b - d;
      if (dm < -(a - c) || dm > (a - c)) return {0.0, 0.0};
      return cscale(cconj(hget(X, a - c, dm)), ldexp(1.0, -c));
    }
    // L2L: out (j = a, i = b), in (k = c, l = d)
    if (c < a) return {0.0, 0.0};
    int dl = d - b;
    if (dl < -(c - a) || dl > (c - a)) return {0.0, 0.0};
    return cscale(cconj(hget(X, c - a, dl)), ldexp(1.0, -(a + 1)));
  }
};

template <class R>
__device__ __forceinline__ void put(R* op, int Kp, bool out_major, int ro, int ri, double v, int* range_bad) {
  if (out_major) op[(int64_t)ro * Kp + ri] = (R)v;
  else op[(int64_t)ri * Kp + ro] = (R)v;
  if (sizeof(R) == 4 && !(fabs(v) <= (double)FLT_MAX)) *range_bad = 1;
}

// Real Kp x Kp matrices of one operator per blockIdx.x; the gridDim.y blocks
// of an operator split its entries (each forms the harmonics X in shared
// memory).  geom: per operator (x, y, z, log2(R_A / r), log2(R_B / r)) in
// double.  Every entry of the K x K corner is written once, so the blocks
// zero only the padding and need no ordering among themselves.
template <class R>
__global__ void k_build_ops(int kind, int p, int Kp, const double* __restrict__ geom, int nops,
                            R* __restrict__ ops, float* __restrict__ ops_lo, bool out_major,
                            int* __restrict__ range_bad) {
  extern __shared__ cd X[];
  __shared__ double scale[kMaxP * kMaxP];
  const int op = blockIdx.x;
  if (op >= nops) return;
  const double* g = geom + 5 * (int64_t)op;
  const int P = kind == kM2L ? 2 * p - 1 : p;
  const int eA = (int)g[3], eB = (int)g[4];
  if (kind == kM2L) irregular_tri(g[0], g[1], g[2], P, X);
  else regular_tri(g[0], g[1], g[2], P, X);
  // the M2L scale factors, one exponent per (output degree, input degree)
  for (int w = threadIdx.x; w < kMaxP * kMaxP; w += blockDim.x) {
    const int a = w / kMaxP, c = w % kMaxP;
    scale[w] = ldexp((a & 1) ? -1.0 : 1.0, eB * (a + 1) + eA * c);
  }
  __syncthreads();
  Coef C{kind, eA, eB, X, scale};
  R* o = ops + (int64_t)op * Kp * Kp;
  float* olo = ops_lo ? ops_lo + (int64_t)op * Kp * Kp : nullptr;
  // the padding rows and columns (index >= K) are zero
  const int K = p * p, part = blockIdx.y, nparts = gridDim.y;
  for (int i = threadIdx.x + part * blockDim.x; i < Kp * Kp; i += blockDim.x * nparts) {
    if (i / Kp < K && i % Kp < K) continue;
    o[i] = (R)0;
    if (olo) olo[i] = 0.0f;
  }
  const int nt = p * (p + 1) / 2;
  for (int w = threadIdx.x + part * blockDim.x; w < nt * nt; w += blockDim.x * nparts) {
    const int oi = w / nt, ii = w % nt;
    int a = 0;
    while ((a + 1) * (a + 2) / 2 <= oi) ++a;
    const int b = oi - a * (a + 1) / 2;
    int c = 0;
    while ((c + 1) * (c + 2) / 2 <= ii) ++c;
    const int d = ii - c * (c + 1) / 2;
    double vals[4];  // (Re out, Im out) x (Re in, Im in)
    if (d == 0) {
      cd cp = C(a, b, c, 0);
      vals[0] = cp.re;
      vals[1] = 0.0;
      vals[2] = cp.im;
      vals[3] = 0.0;
    } else {
      cd cp = C(a, b, c, d), cn = C(a, b, c, -d);
      const double s = (d & 1) ? -1.0 : 1.0;
      // input M = u + i v:  cp M + cn (-1)^d conj(M)
      vals[0] = cp.re + s * cn.re;   // Re out <- u
      vals[1] = -cp.im + s * cn.im;  // Re out <- v
      vals[2] = cp.im + s * cn.im;   // Im out <- u
      vals[3] = cp.re - s * cn.re;   // Im out <- v
    }
    const int nout = b == 0 ? 1 : 2, nin = d == 0 ? 1 : 2;
    for (int po = 0; po < nout; ++po)
      for (int pi = 0; pi < nin; ++pi) {
        const double v = vals[2 * po + pi];
        const int ro = ridx(a, b, po), ri = ridx(c, d, pi);
        put<R>(o, Kp, out_major, ro, ri, v, range_bad);
        if (olo) {
          // 3xTF32 split: hi rounded to TF32 (round to nearest), lo the rest
          float hf = (float)v;
          uint32_t hb;
          asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(hf));
          float hi = __uint_as_float(hb);
          // the low part rounded to TF32 as well, so the tensor core sees it
          // exactly (its own conversion would truncate)
          float lo;
          {
            uint32_t lb;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lb) : "f"((float)(v - (double)hi)));
            lo = __uint_as_float(lb);
          }
          int64_t at = out_major ? (int64_t)ro * Kp + ri : (int64_t)ri * Kp + ro;
          o[at] = (R)hi;
          olo[at] = lo;
        }
      }
  }
}

// ------------------------------------------------------------- M2L plan
struct CellView {
  const int32_t *level, *ix, *iy, *iz;
};

// Targets ordered by (level, octant within the parent, level-difference
// signature, boundary pattern, cell).  The pattern is, per axis, how many
// cells (up to kPatternReach) the domain still holds below and above the
// cell: interior cells and cells at the same place on the boundary have the
// same set of translation offsets, so tiles of them need fewer distinct
// operators (fewer, fuller entries).
// Between octant and pattern the key holds the target's level-difference
// signature (which of source level below / equal / above its own occur
// among its M2L sources): in adaptive trees the cross-level classes follow
// the refinement around a cell, and grouping by it raises Plummer's slot use
// from 0.64 to 0.75 (uniform trees have one signature and keep their order).
// The cell goes with the key as the value of a stable sort whose input is in
// cell order, which orders equal keys by cell.  Cells that take no M2L get
// key 2^kTargetKeyBits (last).
constexpr int kPatternReach = 4;
constexpr int kPatternBits = 14;  // (reach + 1)^6 = 15625 patterns < 2^14
constexpr int kTargetKeyBits = 5 + 3 + 3 + kPatternBits;  // level, octant, signature, pattern

__global__ void k_target_keys(const int32_t* __restrict__ has, CellView c, int ncell, uint64_t* __restrict__ key,
                              int32_t* __restrict__ cell) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ncell) return;
  cell[i] = i;
  if (has[i]) {
    const int l = c.level[i];
    const int side = (1 << l) - 1;
    const int co[3] = {c.ix[i], c.iy[i], c.iz[i]};
    uint64_t pat = 0;
    for (int d = 0; d < 3; ++d) {
      const int lo = min(co[d], kPatternReach), hi = min(side - co[d], kPatternReach);
      pat = pat * ((kPatternReach + 1) * (kPatternReach + 1)) + (uint64_t)(lo * (kPatternReach + 1) + hi);
    }
    const uint64_t oct = ((co[0] & 1) << 2) | ((co[1] & 1) << 1) | (co[2] & 1);
    const uint64_t sig = (uint64_t)(has[i] & 7);
    key[i] = ((uint64_t)l << (6 + kPatternBits)) | (oct << (3 + kPatternBits)) | (sig << kPatternBits) | pat;
  } else {
    key[i] = 1ull << kTargetKeyBits;
  }
}

__global__ void k_target_rank(const int32_t* __restrict__ sorted_cell, int64_t ntgt, int64_t padded,
                              int32_t* __restrict__ tile_tgt, int32_t* __restrict__ rank_of) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= padded) return;
  if (r < ntgt) {
    const int cell = sorted_cell[r];
    tile_tgt[r] = cell;
    rank_of[cell] = (int32_t)r;
  } else {
    tile_tgt[r] = -1;
  }
}

__device__ __forceinline__ void pair_offset(const CellView& c, int A, int B, int64_t d[3], int& dl) {
  const int la = c.level[A], lb = c.level[B];
  const int lmax = la > lb ? la : lb;
  const int sh = kMaxLevel - lmax;
  d[0] = (((2ll * c.ix[A] + 1) << (kMaxLevel - la)) - ((2ll * c.ix[B] + 1) << (kMaxLevel - lb))) >> sh;
  d[1] = (((2ll * c.iy[A] + 1) << (kMaxLevel - la)) - ((2ll * c.iy[B] + 1) << (kMaxLevel - lb))) >> sh;
  d[2] = (((2ll * c.iz[A] + 1) << (kMaxLevel - la)) - ((2ll * c.iz[B] + 1) << (kMaxLevel - lb))) >> sh;
  dl = la - lb;
}

// Class key of a pair: (level difference, offset in units of the smaller
// cell's half side), packed into 6 + 3 b bits with every offset component
// biased by maxd.  Offsets too large for 63 bits (b > 19) get a key of their
// own (top bit set, then the pair index).
__global__ void k_class_keys(const int32_t* __restrict__ tgt, const int32_t* __restrict__ src,
                             int64_t n, CellView c, int b, int64_t maxd, uint64_t* __restrict__ key,
                             int32_t* __restrict__ val) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t d[3];
  int dl;
  pair_offset(c, src[i], tgt[i], d, dl);
  if (b <= 19) {
    key[i] = ((uint64_t)(dl + kMaxLevel) << (3 * b)) | ((uint64_t)(d[0] + maxd) << (2 * b)) |
             ((uint64_t)(d[1] + maxd) << b) | (uint64_t)(d[2] + maxd);
  } else {
    key[i] = (1ull << 63) | (uint64_t)i;
  }
  val[i] = (int32_t)i;
}

__global__ void k_unique_flags(const uint64_t* __restrict__ key, int64_t n, int shift,
                               int64_t* __restrict__ f) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  f[i] = (i == 0 || (key[i] >> shift) != (key[i - 1] >> shift)) ? 1 : 0;
}

// Class id of every pair and the descriptor (dl, dx, dy, dz) of every class.
__global__ void k_class_assign(const uint64_t* __restrict__ key, const int32_t* __restrict__ val,
                               const int64_t* __restrict__ excl, int64_t n,
                               const int32_t* __restrict__ tgt, const int32_t* __restrict__ src,
                               CellView c, int32_t* __restrict__ class_of, int32_t* __restrict__ desc) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool first = i == 0 || key[i] != key[i - 1];
  const int64_t cid = excl[i] + (first ? 0 : -1);
  class_of[val[i]] = (int32_t)cid;
  if (!first) return;
  const int pi = val[i];
  const int A = src[pi], B = tgt[pi];
  const int la = c.level[A], lb = c.level[B];
  const int lmax = la > lb ? la : lb;
  const int sh = kMaxLevel - lmax;
  desc[4 * cid + 0] = la - lb;
  desc[4 * cid + 1] = (int32_t)((((2ll * c.ix[A] + 1) << (kMaxLevel - la)) - ((2ll * c.ix[B] + 1) << (kMaxLevel - lb))) >> sh);
  desc[4 * cid + 2] = (int32_t)((((2ll * c.iy[A] + 1) << (kMaxLevel - la)) - ((2ll * c.iy[B] + 1) << (kMaxLevel - lb))) >> sh);
  desc[4 * cid + 3] = (int32_t)((((2ll * c.iz[A] + 1) << (kMaxLevel - la)) - ((2ll * c.iz[B] + 1) << (kMaxLevel - lb))) >> sh);
}

// Entry key of a pair: (target tile, class, tile row) in tb + cb + 7 bits.
__global__ void k_entry_keys(const int32_t* __restrict__ tgt, const int32_t* __restrict__ src,
                             const int32_t* __restrict__ class_of, const int32_t* __restrict__ rank_of,
                             int64_t n, int cb, uint64_t* __restrict__ key, int32_t* __restrict__ val) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t r = (uint64_t)rank_of[tgt[i]];
  const uint64_t tile = r / kTile, slot = r % kTile;
  key[i] = (tile << (cb + 7)) | ((uint64_t)(uint32_t)class_of[i] << 7) | slot;
  val[i] = src[i];
}

__global__ void k_entry_fill(const uint64_t* __restrict__ key, const int32_t* __restrict__ val,
                             const int64_t* __restrict__ excl, int64_t n, int cb, int32_t* __restrict__ entry_class,
                             int32_t* __restrict__ entry_src, uint64_t* __restrict__ entry_key) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool first = i == 0 || (key[i] >> 7) != (key[i - 1] >> 7);
  const int64_t e = excl[i] + (first ? 0 : -1);
  entry_src[e * kTile + (key[i] & (kTile - 1))] = val[i];
  if (first) {
    entry_class[e] = (int32_t)((key[i] >> 7) & ((1ull << cb) - 1));
    entry_key[e] = key[i] >> (cb + 7);  // tile
  }
}

__global__ void k_tile_ptr(const uint64_t* __restrict__ etile, int64_t ne, int ntile,
                           int32_t* __restrict__ ptr) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t > ntile) return;
  int64_t lo = 0, hi = ne;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (etile[mid] < (uint64_t)t) lo = mid + 1;
    else hi = mid;
  }
  ptr[t] = (int32_t)lo;
}

// Dense form of the class and entry numbering, used when the key space is
// small: a table over all possible keys marks the keys present, and the
// exclusive scan of the marks numbers them in ascending key order, which is
// the numbering the sort-and-unique form produces.
__device__ __forceinline__ uint64_t class_key(const CellView& c, int A, int B, int b, int64_t maxd) {
  int64_t d[3];
  int dl;
  pair_offset(c, A, B, d, dl);
  return ((uint64_t)(dl + kMaxLevel) << (3 * b)) | ((uint64_t)(d[0] + maxd) << (2 * b)) |
         ((uint64_t)(d[1] + maxd) << b) | (uint64_t)(d[2] + maxd);
}

// Marks the class key of every pair in the dense table and keeps the key per
// pair (the entry passes then read it instead of gathering both cells again).
__global__ void k_class_mark(const int32_t* __restrict__ tgt, const int32_t* __restrict__ src, int64_t n,
                             CellView c, int b, int64_t maxd, int64_t* __restrict__ mark,
                             uint32_t* __restrict__ pkey) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t k = class_key(c, src[i], tgt[i], b, maxd);
  pkey[i] = (uint32_t)k;
  // read first: 16.8 M pairs share a few hundred classes, so almost every
  // pair finds its mark set and stores nothing (a plain store from every
  // pair contends for those few addresses)
  if (mark[k] == 0) mark[k] = 1;
}

// The same from the traversal's packed class offsets (no gathers of the
// cells); used while every offset stays within +-127.
__global__ void k_class_mark_packed(const uint32_t* __restrict__ off, int64_t n, int b, int64_t maxd,
                                    int64_t* __restrict__ mark, uint32_t* __restrict__ pkey) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t w = off[i];
  const int64_t dl = (int64_t)(w >> 24) - 32;
  const int64_t d0 = (int8_t)(w >> 16), d1 = (int8_t)(w >> 8), d2 = (int8_t)w;
  const uint64_t k = ((uint64_t)(dl + kMaxLevel) << (3 * b)) | ((uint64_t)(d0 + maxd) << (2 * b)) |
                     ((uint64_t)(d1 + maxd) << b) | (uint64_t)(d2 + maxd);
  pkey[i] = (uint32_t)k;
  if (mark[k] == 0) mark[k] = 1;
}

// After the scan: class id of every pair.
__global__ void k_class_lookup(const int32_t* __restrict__ tgt, const int32_t* __restrict__ src, int64_t n,
                               CellView c, int b, int64_t maxd, const int64_t* __restrict__ excl,
                               int32_t* __restrict__ class_of) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  class_of[i] = (int32_t)excl[class_key(c, src[i], tgt[i], b, maxd)];
}

// Descriptor (dl, dx, dy, dz) of every class, decoded from its key.
__global__ void k_class_desc_dense(const int64_t* __restrict__ excl, int64_t nkey, int64_t total, int b,
                                   int64_t maxd, int32_t* __restrict__ desc) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= nkey) return;
  const int64_t next = k + 1 < nkey ? excl[k + 1] : total;
  if (next == excl[k]) return;  // key absent
  const int64_t cid = excl[k];
  const uint64_t m = (1ull << b) - 1;
  desc[4 * cid + 0] = (int32_t)((int64_t)((uint64_t)k >> (3 * b)) - kMaxLevel);
  desc[4 * cid + 1] = (int32_t)((int64_t)(((uint64_t)k >> (2 * b)) & m) - maxd);
  desc[4 * cid + 2] = (int32_t)((int64_t)(((uint64_t)k >> b) & m) - maxd);
  desc[4 * cid + 3] = (int32_t)((int64_t)((uint64_t)k & m) - maxd);
}

// Class of pair i: from the per-pair array of the sorted numbering, or
// looked up in the scanned dense key table.
struct ClassOf {
  const int32_t* class_of;  // sorted numbering, else null
  const int64_t* key_excl;  // dense numbering: scanned key table
  const uint32_t* pkey;     // dense numbering: the class key of every pair
  __device__ __forceinline__ int operator()(int64_t i) const {
    if (class_of) return class_of[i];
    return (int)key_excl[pkey[i]];
  }
};

__global__ void k_entry_mark(const int32_t* __restrict__ tgt, const int32_t* __restrict__ src, ClassOf cls,
                             const int32_t* __restrict__ rank_of, int64_t n, int nclass,
                             int64_t* __restrict__ mark) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int t = tgt[i];
  const int64_t e = (int64_t)(rank_of[t] / kTile) * nclass + cls(i);
  mark[e] = 1;  // plain store: the entries are many, each marked by at most 128 pairs
}

__global__ void k_entry_fill_dense(const int32_t* __restrict__ tgt, const int32_t* __restrict__ src, ClassOf cls,
                                   const int32_t* __restrict__ rank_of, int64_t n, int nclass,
                                   const int64_t* __restrict__ excl, int32_t* __restrict__ entry_src) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int t = tgt[i], sr = src[i];
  const int r = rank_of[t];
  const int64_t e = excl[(int64_t)(r / kTile) * nclass + cls(i)];
  entry_src[e * kTile + (r % kTile)] = sr;
}

// Entry classes and tile pointers from the scanned (tile, class) table.
__global__ void k_entry_table(const int64_t* __restrict__ excl, int ntile, int nclass, int64_t total,
                              int32_t* __restrict__ entry_class, int32_t* __restrict__ tile_eptr) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nk = (int64_t)ntile * nclass;
  if (k > nk) return;
  if (k == nk) {
    tile_eptr[ntile] = (int32_t)total;
    return;
  }
  if (k % nclass == 0) tile_eptr[k / nclass] = (int32_t)excl[k];
  const int64_t next = k + 1 < nk ? excl[k + 1] : total;
  if (next != excl[k]) entry_class[excl[k]] = (int32_t)(k % nclass);
}

__global__ void k_m2l_geom(const int32_t* __restrict__ desc, int n, double* __restrict__ geom) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int dl = desc[4 * i];
  // (c_B - c_A) / r = -(dx, dy, dz); R_A / r = 2^max(0, -dl), R_B / r = 2^max(0, dl)
  geom[5 * i + 0] = -(double)desc[4 * i + 1];
  geom[5 * i + 1] = -(double)desc[4 * i + 2];
  geom[5 * i + 2] = -(double)desc[4 * i + 3];
  geom[5 * i + 3] = dl < 0 ? -dl : 0;  // log2(R_A / r)
  geom[5 * i + 4] = dl > 0 ? dl : 0;   // log2(R_B / r)
}

// Single-precision M2L operators (the same entries as k_build_ops).  FP64
// runs at a small fraction of the FP32 rate on this GPU, so only the
// harmonics are computed in double (a thread per column, as above); each is then held
// as a pair of floats (hi + lo, about 48 bits), and the per-entry work -- the
// sum of the +m and -m parts, the power-of-two scale and the TF32 split --
// runs in FP32 on those pairs.  A pair's low part that underflows only drops
// digits below 2^-126 of the operator.
struct ff {
  float h, l;
};
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const float s = a.h + b.h;
  const float bb = s - a.h;
  float e = (a.h - (s - bb)) + (b.h - bb);
  e += a.l + b.l;
  const float h = s + e;
  return ff{h, e - (h - s)};
}
__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.h, -a.l}; }

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t b;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(b) : "f"(x));
  return __uint_as_float(b);
}

__global__ void k_build_m2l_f32(int p, int Kp, const double* __restrict__ geom, int nops, float* __restrict__ ops,
                                float* __restrict__ ops_lo, int* __restrict__ range_bad) {
  extern __shared__ cd X[];  // the (2p - 1)-degree triangle, then its float pairs
  const int op = blockIdx.x;
  if (op >= nops) return;
  const double* g = geom + 5 * (int64_t)op;
  const int P = 2 * p - 1;
  const int ntri = P * (P + 1) / 2;
  float4* Xf = reinterpret_cast<float4*>(X + ntri);  // (re hi, re lo, im hi, im lo)
  const int eA = (int)g[3], eB = (int)g[4];
  irregular_tri(g[0], g[1], g[2], P, X);
  float* o = ops + (int64_t)op * Kp * Kp;
  float* olo = ops_lo ? ops_lo + (int64_t)op * Kp * Kp : nullptr;
  for (int i = threadIdx.x; i < Kp * Kp; i += blockDim.x) {
    o[i] = 0.0f;
    if (olo) olo[i] = 0.0f;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < ntri; k += blockDim.x) {
    const double re = X[k].re, im = X[k].im;
    const float rh = (float)re, ih = (float)im;
    Xf[k] = make_float4(rh, (float)(re - (double)rh), ih, (float)(im - (double)ih));
  }
  __syncthreads();
  const int nt = p * (p + 1) / 2;
  for (int w = threadIdx.x; w < nt * nt; w += blockDim.x) {
    const int oi = w / nt, ii = w % nt;
    int a = 0;
    while ((a + 1) * (a + 2) / 2 <= oi) ++a;
    const int b = oi - a * (a + 1) / 2;
    int c = 0;
    while ((c + 1) * (c + 2) / 2 <= ii) ++c;
    const int d = ii - c * (c + 1) / 2;
    const int n = a + c;
    // X_n^m for -n <= m <= n (X_n^{-m} = (-1)^m conj(X_n^m))
    auto get = [&](int m, ff& re, ff& im) {
      const float4 v = Xf[tri(n, m < 0 ? -m : m)];
      re = ff{v.x, v.y};
      im = ff{v.z, v.w};
      if (m < 0) {
        im = ff_neg(im);
        if ((-m) & 1) {
          re = ff_neg(re);
          im = ff_neg(im);
        }
      }
    };
    ff vals[4];  // (Re out, Im out) x (Re in, Im in)
    ff pr, pi;
    get(d + b, pr, pi);
    if (d == 0) {
      vals[0] = pr;
      vals[1] = ff{0.f, 0.f};
      vals[2] = pi;
      vals[3] = ff{0.f, 0.f};
    } else {
      ff nr, ni;
      get(b - d, nr, ni);
      if (d & 1) {
        nr = ff_neg(nr);
        ni = ff_neg(ni);
      }
      // input M = u + i v:  cp M + cn (-1)^d conj(M)
      vals[0] = ff_add(pr, nr);
      vals[1] = ff_add(ff_neg(pi), ni);
      vals[2] = ff_add(pi, ni);
      vals[3] = ff_add(pr, ff_neg(nr));
    }
    // (-1)^a 2^(eB (a + 1) + eA c), exact in float
    const float sc = ldexpf((a & 1) ? -1.0f : 1.0f, eB * (a + 1) + eA * c);
    const int nout = b == 0 ? 1 : 2, nin = d == 0 ? 1 : 2;
    for (int po = 0; po < nout; ++po)
      for (int q = 0; q < nin; ++q) {
        const ff v = vals[2 * po + q];
        const float h = v.h * sc, l = v.l * sc;
        if (!(fabsf(h) <= FLT_MAX)) *range_bad = 1;
        const int64_t at = (int64_t)ridx(a, b, po) * Kp + ridx(c, d, q);
        if (olo) {
          const float hi = tf32_rna(h);
          o[at] = hi;
          olo[at] = tf32_rna((h - hi) + l);
        } else {
          o[at] = h + l;
        }
      }
  }
}

}  // namespace

void build_m2l_plan(fmm_tree* t) {
  Arena& a = t->arena;
  cudaStream_t s = t->stream;
  const int64_t nm = t->n_m2l;
  CellView cv{t->c.level, t->c.ix, t->c.iy, t->c.iz};
  if (nm == 0) {
    t->nclass = 0;
    t->ntile = 0;
    t->nentry = 0;
    t->tile_eptr = alloc_n<int32_t>(a, 1);
    GB_CK(cudaMemsetAsync(t->tile_eptr, 0, sizeof(int32_t), s));
    return;
  }
  // --- targets and tiles (the traversal marked the cells that take M2L and
  // found the largest class offset)
  int32_t* has = t->m2l_has;
  uint64_t* tkey = alloc_n<uint64_t>(a, t->ncell);
  int32_t* tcell = alloc_n<int32_t>(a, t->ncell);
  k_target_keys<<<blocks(t->ncell), kThreads, 0, s>>>(has, cv, t->ncell, tkey, tcell);
  GB_LAUNCH("k_target_keys");
  radix_sort_pairs(a, tkey, tcell, t->ncell, kTargetKeyBits + 1, s);
  // the target count and the largest class offset came with the traversal
  const unsigned long long ntgt = (unsigned long long)t->m2l_ntgt, maxd = t->m2l_maxd_host;
  t->ntile = (int)((ntgt + kTile - 1) / kTile);
  const int64_t padded = (int64_t)t->ntile * kTile;
  t->tile_tgt = alloc_n<int32_t>(a, padded);
  int32_t* rank_of = alloc_n<int32_t>(a, t->ncell);
  k_target_rank<<<blocks(padded), kThreads, 0, s>>>(tcell, (int64_t)ntgt, padded, t->tile_tgt, rank_of);
  GB_LAUNCH("k_target_rank");
  a.release(tkey);
  a.release(tcell);

  // --- translation classes
  int b = 1;
  while ((1ull << b) <= 2 * maxd) ++b;
  // dense numbering while the key table stays small (2^22 keys), else sort
  const int kbits = 6 + 3 * b;
  const bool sorted_only = (t->flags & FMM_FLAG_SORTED_PLAN) != 0;
  const bool dense_cls = !sorted_only && b <= 19 && kbits <= kDenseBits;
  int32_t* class_of = nullptr;
  int64_t* key_excl = nullptr;  // dense numbering: kept for the entry kernels
  uint32_t* pkey = nullptr;     // dense numbering: class key per pair
  if (dense_cls) {
    const int64_t nkey = 1ll << kbits;
    key_excl = alloc_n<int64_t>(a, nkey);
    pkey = alloc_n<uint32_t>(a, nm);
    GB_CK(cudaMemsetAsync(key_excl, 0, sizeof(int64_t) * nkey, s));
    if (t->m2l_off && maxd <= 127) {
      k_class_mark_packed<<<blocks(nm), kThreads, 0, s>>>(t->m2l_off, nm, b, (int64_t)maxd, key_excl, pkey);
      GB_LAUNCH("k_class_mark_packed");
    } else {
      k_class_mark<<<blocks(nm), kThreads, 0, s>>>(t->m2l_tgt, t->m2l_src, nm, cv, b, (int64_t)maxd, key_excl,
                                                   pkey);
      GB_LAUNCH("k_class_mark");
    }
    const int64_t ncls = scan_exclusive_i64_total(a, key_excl, nkey, s);
    t->nclass = (int)ncls;
    t->class_desc = alloc_n<int32_t>(a, 4 * ncls);
    k_class_desc_dense<<<blocks(nkey), kThreads, 0, s>>>(key_excl, nkey, ncls, b, (int64_t)maxd, t->class_desc);
    GB_LAUNCH("k_class_desc_dense");
  } else {
    uint64_t* ckey = alloc_n<uint64_t>(a, nm);
    int32_t* cval = alloc_n<int32_t>(a, nm);
    k_class_keys<<<blocks(nm), kThreads, 0, s>>>(t->m2l_tgt, t->m2l_src, nm, cv, b, (int64_t)maxd, ckey, cval);
    GB_LAUNCH("k_class_keys");
    radix_sort_pairs(a, ckey, cval, nm, b <= 19 ? 6 + 3 * b : 64, s);
    int64_t* flag = alloc_n<int64_t>(a, nm);
    k_unique_flags<<<blocks(nm), kThreads, 0, s>>>(ckey, nm, 0, flag);
    GB_LAUNCH("k_unique_flags");
    const int64_t ncls = scan_exclusive_i64_total(a, flag, nm, s);
    if (ncls > 0x7fffffff) fail(FMM_ERR_ARG, "too many translation classes");
    t->nclass = (int)ncls;
    t->class_desc = alloc_n<int32_t>(a, 4 * ncls);
    class_of = alloc_n<int32_t>(a, nm);
    k_class_assign<<<blocks(nm), kThreads, 0, s>>>(ckey, cval, flag, nm, t->m2l_tgt, t->m2l_src, cv,
                                                   class_of, t->class_desc);
    GB_LAUNCH("k_class_assign");
    a.release(ckey);
    a.release(cval);
    a.release(flag);
  }

  // --- entries: (tile, class) with the source of every tile row
  if (!sorted_only && (int64_t)t->ntile * t->nclass <= (1ll << kDenseBits)) {
    const int64_t nk = (int64_t)t->ntile * t->nclass;
    int64_t* mark = alloc_n<int64_t>(a, nk);
    GB_CK(cudaMemsetAsync(mark, 0, sizeof(int64_t) * nk, s));
    const ClassOf cls{class_of, key_excl, pkey};
    k_entry_mark<<<blocks(nm), kThreads, 0, s>>>(t->m2l_tgt, t->m2l_src, cls, rank_of, nm, t->nclass, mark);
    GB_LAUNCH("k_entry_mark");
    const int64_t ne = scan_exclusive_i64_total(a, mark, nk, s);
    t->nentry = ne;
    t->entry_class = alloc_n<int32_t>(a, ne);
    t->entry_src = alloc_n<int32_t>(a, ne * kTile);
    GB_CK(cudaMemsetAsync(t->entry_src, 0xff, sizeof(int32_t) * ne * kTile, s));
    k_entry_fill_dense<<<blocks(nm), kThreads, 0, s>>>(t->m2l_tgt, t->m2l_src, cls, rank_of, nm, t->nclass, mark,
                                                       t->entry_src);
    GB_LAUNCH("k_entry_fill_dense");
    t->tile_eptr = alloc_n<int32_t>(a, t->ntile + 1);
    k_entry_table<<<blocks(nk + 1), kThreads, 0, s>>>(mark, t->ntile, t->nclass, ne, t->entry_class,
                                                      t->tile_eptr);
    GB_LAUNCH("k_entry_table");
    a.release(mark);
    if (class_of) a.release(class_of);
    if (key_excl) a.release(key_excl);
    if (pkey) a.release(pkey);
    a.release(rank_of);
    return;
  }
  if (pkey) a.release(pkey);
  if (!class_of) {
    // dense class numbering, sorted entries: the per-pair classes
    class_of = alloc_n<int32_t>(a, nm);
    k_class_lookup<<<blocks(nm), kThreads, 0, s>>>(t->m2l_tgt, t->m2l_src, nm, cv, b, (int64_t)maxd, key_excl,
                                                   class_of);
    GB_LAUNCH("k_class_lookup");
  }
  if (key_excl) a.release(key_excl);
  uint64_t* ekey = alloc_n<uint64_t>(a, nm);
  int32_t* eval = alloc_n<int32_t>(a, nm);
  int cb = 1, tb = 1;
  while ((1ll << cb) < (int64_t)t->nclass) ++cb;
  while ((1ll << tb) < (int64_t)t->ntile) ++tb;
  if (tb + cb + 7 > 64) fail(FMM_ERR_ARG, "M2L plan key too wide");
  k_entry_keys<<<blocks(nm), kThreads, 0, s>>>(t->m2l_tgt, t->m2l_src, class_of, rank_of, nm, cb, ekey, eval);
  GB_LAUNCH("k_entry_keys");
  a.release(class_of);
  a.release(rank_of);
  radix_sort_pairs(a, ekey, eval, nm, tb + cb + 7, s);
  int64_t* eflag = alloc_n<int64_t>(a, nm);
  k_unique_flags<<<blocks(nm), kThreads, 0, s>>>(ekey, nm, 7, eflag);
  GB_LAUNCH("k_unique_flags");
  const int64_t ne = scan_exclusive_i64_total(a, eflag, nm, s);
  t->nentry = ne;
  t->entry_class = alloc_n<int32_t>(a, ne);
  t->entry_src = alloc_n<int32_t>(a, ne * kTile);
  GB_CK(cudaMemsetAsync(t->entry_src, 0xff, sizeof(int32_t) * ne * kTile, s));
  uint64_t* etile = alloc_n<uint64_t>(a, ne);
  k_entry_fill<<<blocks(nm), kThreads, 0, s>>>(ekey, eval, eflag, nm, cb, t->entry_class, t->entry_src, etile);
  GB_LAUNCH("k_entry_fill");
  t->tile_eptr = alloc_n<int32_t>(a, t->ntile + 1);
  k_tile_ptr<<<blocks(t->ntile + 1), kThreads, 0, s>>>(etile, ne, t->ntile, t->tile_eptr);
  GB_LAUNCH("k_tile_ptr");
  a.release(ekey);
  a.release(eval);
  a.release(eflag);
  a.release(etile);
}

void build_operators(fmm_tree* t) {
  Arena& a = t->arena;
  cudaStream_t s = t->stream;
  const bool f64 = t->precision == 64;
  const size_t rs = f64 ? sizeof(double) : sizeof(float);
  const int p = t->p, Kp = t->Kp;
  // an operator entry out of the float range sets this flag; it is read back
  // at the end of the build (FMM_ERR_RANGE)
  int* bad = reinterpret_cast<int*>(t->d_tail + 2);
  // M2M / L2L: 8 octants, child offset (c_C - c_P)/R_P = (bx, by, bz) - 1/2
  double hgeom[8 * 5];
  for (int o = 0; o < 8; ++o) {
    hgeom[5 * o + 0] = ((o >> 2) & 1) - 0.5;
    hgeom[5 * o + 1] = ((o >> 1) & 1) - 0.5;
    hgeom[5 * o + 2] = (o & 1) - 0.5;
    hgeom[5 * o + 3] = 0.0;
    hgeom[5 * o + 4] = 0.0;
  }
  double* g8 = alloc_n<double>(a, 40);
  GB_CK(cudaMemcpyAsync(g8, hgeom, sizeof(hgeom), cudaMemcpyHostToDevice, s));
  t->m2m_ops = a.alloc(rs * 8 * Kp * Kp);
  t->l2l_ops = a.alloc(rs * 8 * Kp * Kp);
  const size_t sm_reg = sizeof(double) * 2 * (size_t)p * (p + 1) / 2;
  const int Pt = 2 * p - 1;
  const size_t sm_irr = sizeof(double) * 2 * (size_t)Pt * (Pt + 1) / 2;
  // 8 octant operators each, their entries split over 16 blocks (the FP64
  // pipe of 8 SMs alone took 60 us per set at p = 10)
  const dim3 g8x16(8, 16);
  if (f64) {
    k_build_ops<double><<<g8x16, 256, sm_reg, s>>>(kM2M, p, Kp, g8, 8, (double*)t->m2m_ops, nullptr, false, bad);
    k_build_ops<double><<<g8x16, 256, sm_reg, s>>>(kL2L, p, Kp, g8, 8, (double*)t->l2l_ops, nullptr, false, bad);
  } else {
    k_build_ops<float><<<g8x16, 256, sm_reg, s>>>(kM2M, p, Kp, g8, 8, (float*)t->m2m_ops, nullptr, false, bad);
    k_build_ops<float><<<g8x16, 256, sm_reg, s>>>(kL2L, p, Kp, g8, 8, (float*)t->l2l_ops, nullptr, false, bad);
  }
  GB_LAUNCH("k_build_ops m2m/l2l");
  if (t->nclass > 0) {
    double* geom = alloc_n<double>(a, 5 * (size_t)t->nclass);
    k_m2l_geom<<<blocks(t->nclass), kThreads, 0, s>>>(t->class_desc, t->nclass, geom);
    GB_LAUNCH("k_m2l_geom");
    t->m2l_ops = a.alloc(rs * (size_t)t->nclass * Kp * Kp);
    if (f64) {
      k_build_ops<double><<<t->nclass, 256, sm_irr, s>>>(kM2L, p, Kp, geom, t->nclass, (double*)t->m2l_ops,
                                                         nullptr, true, bad);
    } else {
      if (t->m2l_engine == 1) t->m2l_ops_lo = alloc_n<float>(a, (size_t)t->nclass * Kp * Kp);
      const size_t sm_f = sm_irr + sizeof(float4) * (size_t)Pt * (Pt + 1) / 2;
      k_build_m2l_f32<<<t->nclass, 256, sm_f, s>>>(p, Kp, geom, t->nclass, (float*)t->m2l_ops, t->m2l_ops_lo, bad);
    }
    GB_LAUNCH("k_build_ops m2l");
    a.release(geom);
  }
  a.release(g8);
}

}  // namespace gbfmm
