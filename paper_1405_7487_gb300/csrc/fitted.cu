// fitted.cu -- the far field about particle-fitted centres
// (FMM_FLAG_FITTED_CENTRES).
//
// Sec. II.B: the cells of the paper's code are squeezed to fit their
// particles, which lets a cell accept interactions from closer cells.  Here
// every expansion of a cell is taken about the centre of the box of its
// bodies' voxel centres (the integer u_min + u_max + 1 per axis, units of
// H / 2^21; see traverse.cu), so the translation between two cells depends on
// the pair and no operator is shared: M2M and L2L run per child and M2L per
// pair, each forming its solid harmonics on the fly.  The stored expansions
// keep the scaling of the cube cells (M~ = M / R^n, L~ = L R^(n+1), R the
// cube's half side), so P2M and L2P only change their centre:
//   M2M  M~_n^m(P) += sum_{k,l} M~_k^l(C) 2^-k conj(Ups_{n-k}^{m-l}(t)),
//        t = (c_C - c_P) / R_P
//   L2L  L~_j^i(C) += sum_{k,l} L~_k^l(P) 2^-(j+1) conj(Ups_{k-j}^{l-i}(t))
//   M2L  L~_k^l(B) += (-1)^k sum_{n,m} M~_n^m(A) rho_A^n rho_B^(k+1)
//                     Th_{n+k}^{m+l}(d / |d|),   d = c_B - c_A, rho = R / |d|
// (the conventions of ops.cu and expansions.cu).  Single precision cannot
// hold the harmonics of the unit vector as they are (Th_j grows like
// (2j - 1)!!, 3.5e40 at j = 30), so M2L carries Th_j / j! (at most about
// 2^j) and splits (n + k)! = n! k! C(n + k, k):
//   L~_k^l(B) += (-1)^k rho_B^(k+1) k!  sum_n C(n + k, k)
//                sum_m [M~_n^m rho_A^n n!] [Th_{n+k}^{m+l}(u) / (n + k)!],
// each factor within range for p <= 16 (M~_n rho_A^n n! ~ (r_A / |d|)^n and
// L~_k ~ k! rho_B^(k+1) in this normalisation).  Each target sums its sources in a
// fixed order (the M2L list sorted by source), with compensated (Kahan)
// addition across rounds of sources; the results are reproducible.
#include "kernels.cuh"

namespace gbfmm {
namespace {

constexpr int kThreads = 128;
constexpr int kSrcRound = 8;   // M2L sources per round
constexpr int kLB = 4;         // M2L outputs (consecutive orders l of one degree k) per task
constexpr int kTriP = kMaxP * (kMaxP + 1) / 2;

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <class R>
struct cx {
  R re, im;
};
template <class R>
__device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

__device__ __forceinline__ int tri(int n, int m) { return n * (n + 1) / 2 + m; }
__device__ __forceinline__ int ridx(int n, int m, int part) { return n * n + (m == 0 ? 0 : 2 * m - 1 + part); }

// X_n^m for -n <= m <= n from the m >= 0 triangle (X_n^-m = (-1)^m conj(X_n^m)).
template <class R>
__device__ __forceinline__ cx<R> hget(const cx<R>* X, int n, int m) {
  if (m >= 0) return X[tri(n, m)];
  cx<R> v = X[tri(n, -m)];
  v.im = -v.im;
  if ((-m) & 1) {
    v.re = -v.re;
    v.im = -v.im;
  }
  return v;
}

// The m >= 0 coefficients of an expansion of degree < p as complex numbers
// (from the real packing).
template <class R>
__device__ __forceinline__ void unpack_tri(const R* __restrict__ src, int p, cx<R>* out) {
  for (int i = threadIdx.x; i < p * (p + 1) / 2; i += blockDim.x) {
    int n = 0;
    while ((n + 1) * (n + 2) / 2 <= i) ++n;
    const int m = i - n * (n + 1) / 2;
    out[i] = {src[ridx(n, m, 0)], m ? src[ridx(n, m, 1)] : (R)0};
  }
}

// Column m of the regular harmonics of v (degrees m .. P - 1), by one lane:
// Ups_m^m = (-(x + i y))^m / (2^m m!),
// (n+m)(n-m) Ups_n^m = (2n-1) z Ups_{n-1}^m - r^2 Ups_{n-2}^m.
template <class R>
__device__ __forceinline__ void regular_column(R x, R y, R z, int m, int P, cx<R>* U) {
  cx<R> d{(R)1, (R)0};
  for (int k = 1; k <= m; ++k) {
    d = cmul(d, cx<R>{-x, -y});
    d.re /= (R)(2 * k);
    d.im /= (R)(2 * k);
  }
  const R r2 = x * x + y * y + z * z;
  cx<R> a = d, b{(R)0, (R)0};
  for (int n = m; n < P; ++n) {
    U[tri(n, m)] = a;
    const R f = (R)1 / ((R)(n + 1 + m) * (R)(n + 1 - m));
    const cx<R> c{((R)(2 * n + 1) * z * a.re - r2 * b.re) * f, ((R)(2 * n + 1) * z * a.im - r2 * b.im) * f};
    b = a;
    a = c;
  }
}

// Column m of Th_n^m(u) / n! for a unit vector u (degrees m .. P - 1), from
// Th_m^m = -(2m-1) (x + i y) Th_{m-1}^{m-1} and
// Th_n^m = (2n-1) z Th_{n-1}^m - (n+m-1)(n-m-1) Th_{n-2}^m   (|u| = 1),
// divided through by n! (rcp[q] = 1/q, rcp[0] = 0); stored at T[n*n + n + m] together with the order -m
// (Th_n^-m = (-1)^m conj(Th_n^m)).
template <class R>
__device__ __forceinline__ void irregular_column_full(R x, R y, R z, int m, int P, const R* __restrict__ rcp,
                                                      cx<R>* T) {
  cx<R> d{(R)1, (R)0};
  for (int k = 1; k <= m; ++k) {
    d = cmul(d, cx<R>{x, y});
    const R f = -(R)(2 * k - 1) * rcp[k];
    d.re *= f;
    d.im *= f;
  }
  cx<R> a = d, b{(R)0, (R)0};
  for (int n = m; n < P; ++n) {
    T[n * n + n + m] = a;
    if (m) T[n * n + n - m] = (m & 1) ? cx<R>{-a.re, a.im} : cx<R>{a.re, -a.im};
    const R c1 = (R)(2 * n + 1) * z * rcp[n + 1];
    const R c2 = (R)((n + m) * (n - m)) * rcp[n + 1] * rcp[n];  // rcp[0] = 0
    const cx<R> c{c1 * a.re - c2 * b.re, c1 * a.im - c2 * b.im};
    b = a;
    a = c;
  }
}

// Expansion centres: corner + fc * H / 2^21 in double, and as float pairs.
__global__ void k_fit_centres(const int32_t* __restrict__ fc, int ncell, const double* __restrict__ root,
                              double* __restrict__ cen, float* __restrict__ cenf) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const double unit = ldexp(root[9], -kMaxLevel);
  for (int a = 0; a < 3; ++a) {
    const double v = __dadd_rn(root[10 + a], __dmul_rn((double)fc[3 * c + a], unit));
    cen[3 * c + a] = v;
    const float h = (float)v;
    cenf[6 * c + a] = h;
    cenf[6 * c + 3 + a] = (float)(v - (double)h);
  }
}

// M2M: one block per parent cell of a level; the children one at a time.
template <class R>
__global__ void k_m2m_fit(int first, int ncell, const int32_t* __restrict__ cbeg, const int32_t* __restrict__ nch,
                          const int32_t* __restrict__ level, const double* __restrict__ cen,
                          const double* __restrict__ root, int p, int Kp, R* __restrict__ M) {
  __shared__ cx<R> U[kTriP], Mc[kTriP];
  const int cell = first + blockIdx.x;
  if (blockIdx.x >= ncell) return;
  const int n_ch = nch[cell];
  if (n_ch == 0) return;
  const int nt = p * (p + 1) / 2;
  const double RP = ldexp(root[9], -level[cell]);
  cx<R> acc[2] = {{(R)0, (R)0}, {(R)0, (R)0}};
  for (int c = 0; c < n_ch; ++c) {
    const int ch = cbeg[cell] + c;
    __syncthreads();
    if ((int)threadIdx.x < p) {
      const R tx = (R)((cen[3 * ch] - cen[3 * cell]) / RP), ty = (R)((cen[3 * ch + 1] - cen[3 * cell + 1]) / RP),
              tz = (R)((cen[3 * ch + 2] - cen[3 * cell + 2]) / RP);
      regular_column<R>(tx, ty, tz, threadIdx.x, p, U);
    }
    unpack_tri<R>(M + (int64_t)ch * Kp, p, Mc);
    __syncthreads();
    for (int oi = 0; oi < 2; ++oi) {
      const int o = threadIdx.x + oi * blockDim.x;
      if (o >= nt) continue;
      int n = 0;
      while ((n + 1) * (n + 2) / 2 <= o) ++n;
      const int m = o - n * (n + 1) / 2;
      cx<R> s{(R)0, (R)0};
      R h = 1;  // 2^-k
      for (int k = 0; k <= n; ++k, h *= (R)0.5) {
        cx<R> sk{(R)0, (R)0};
        for (int l = max(-k, m - (n - k)); l <= min(k, m + (n - k)); ++l) {
          const cx<R> a = hget(Mc, k, l), u = hget(U, n - k, m - l);  // M conj(U)
          sk.re += a.re * u.re + a.im * u.im;
          sk.im += a.im * u.re - a.re * u.im;
        }
        s.re += h * sk.re;
        s.im += h * sk.im;
      }
      acc[oi].re += s.re;
      acc[oi].im += s.im;
    }
  }
  for (int oi = 0; oi < 2; ++oi) {
    const int o = threadIdx.x + oi * blockDim.x;
    if (o >= nt) continue;
    int n = 0;
    while ((n + 1) * (n + 2) / 2 <= o) ++n;
    const int m = o - n * (n + 1) / 2;
    R* out = M + (int64_t)cell * Kp;
    out[ridx(n, m, 0)] = acc[oi].re;
    if (m) out[ridx(n, m, 1)] = acc[oi].im;
  }
}

// L2L: one block per cell of a level >= 1: L(C) += shift of L(parent).
template <class R>
__global__ void k_l2l_fit(int first, int ncell, const int32_t* __restrict__ parent, const int32_t* __restrict__ level,
                          const double* __restrict__ cen, const double* __restrict__ root, int p, int Kp,
                          R* __restrict__ L) {
  __shared__ cx<R> U[kTriP], Lp[kTriP];
  const int cell = first + blockIdx.x;
  if (blockIdx.x >= ncell) return;
  const int par = parent[cell];
  const int nt = p * (p + 1) / 2;
  const double RP = ldexp(root[9], -level[par]);
  if ((int)threadIdx.x < p) {
    const R tx = (R)((cen[3 * cell] - cen[3 * par]) / RP), ty = (R)((cen[3 * cell + 1] - cen[3 * par + 1]) / RP),
            tz = (R)((cen[3 * cell + 2] - cen[3 * par + 2]) / RP);
    regular_column<R>(tx, ty, tz, threadIdx.x, p, U);
  }
  unpack_tri<R>(L + (int64_t)par * Kp, p, Lp);
  __syncthreads();
  for (int o = threadIdx.x; o < nt; o += blockDim.x) {
    int j = 0;
    while ((j + 1) * (j + 2) / 2 <= o) ++j;
    const int i = o - j * (j + 1) / 2;
    cx<R> s{(R)0, (R)0};
    for (int k = j; k < p; ++k)
      for (int l = max(-k, i - (k - j)); l <= min(k, i + (k - j)); ++l) {
        const cx<R> a = hget(Lp, k, l), u = hget(U, k - j, l - i);  // L conj(U)
        s.re += a.re * u.re + a.im * u.im;
        s.im += a.im * u.re - a.re * u.im;
      }
    const R h = ldexp((R)1, -(j + 1));
    R* out = L + (int64_t)cell * Kp;
    out[ridx(j, i, 0)] += h * s.re;
    if (i) out[ridx(j, i, 1)] += h * s.im;
  }
}

// M2L: one block per target cell with M2L sources (sources [ptr[t], ptr[t+1])
// of the sorted list), kSrcRound sources per round.  The block forms each
// source's harmonics Th_j^i(u) / j! (all orders -j .. j; a thread per order
// column), its multipoles M~_n^m rho_A^n n! (all m) and the target factors in
// shared memory.  Then thread t takes the tasks t, t + kThreads, ... of the
// round, a task being a source slot r and the kLB outputs (k, l0 .. l0 + kLB
// - 1) of one degree, which share each multipole load and a sliding window of
// harmonics, and adds the contributions to its own accumulators
// (compensated).  Slot r takes sources r,
// r + kSrcRound, ... of the target's list, in order, and the slots are summed
// in order at the end, so the results are reproducible.
// In single precision the geometry comes from the integer centres: their
// differences (below 2^22 units of H / 2^21) are exact in FP32, and the cube
// half side R = 2^(21 - level) units, so no FP64 runs per pair.
template <class R, int kSlots>
__global__ void __launch_bounds__(kThreads) k_m2l_fit(const int32_t* __restrict__ ptr, const int32_t* __restrict__ tgt_of,
                                                       const int32_t* __restrict__ src, const int32_t* __restrict__ level,
                                                       const int32_t* __restrict__ fc, const double* __restrict__ cen,
                                                       const double* __restrict__ root, int p, int Kp,
                                                       const R* __restrict__ M, R* __restrict__ L) {
  extern __shared__ unsigned char smem_raw[];
  const int PT = 2 * p - 1, nT = PT * PT, nM = p * p, nt = p * (p + 1) / 2;
  cx<R>* T = reinterpret_cast<cx<R>*>(smem_raw);      // kSrcRound x PT^2, index j*j + j + i
  cx<R>* Mr = T + kSrcRound * nT;                     // kSrcRound x p^2, index n*n + n + m
  R* fk = reinterpret_cast<R*>(Mr + kSrcRound * nM);  // kSrcRound x p: (-1)^k rho_B^(k+1) k!
  R* gA = fk + kSrcRound * p;                         // kSrcRound x p: rho_A^n n!
  R* geo = gA + kSrcRound * p;                        // kSrcRound x 3: d / |d|
  R* bin = geo + kSrcRound * 3;                       // p x p: C(n + k, k) at n * p + k
  R* rcp = bin + p * p;                               // 2 kMaxP: 1 / q (rcp[0] = 0)
  const int tb = tgt_of[blockIdx.x];
  const int e0 = ptr[tb], e1 = ptr[tb + 1];
  for (int i = threadIdx.x; i < p * p; i += kThreads) {
    const int n = i / p, k = i - n * p;
    R c = 1;
    for (int q = 1; q <= k; ++q) c = c * (R)(n + q) / (R)q;
    bin[i] = c;
  }
  if (threadIdx.x < 2 * kMaxP) rcp[threadIdx.x] = threadIdx.x ? (R)1 / (R)threadIdx.x : (R)0;
  // This thread's tasks: slot j is task threadIdx.x + j * kThreads, a
  // (source slot r, row k, outputs l0 .. l0 + kLB - 1) block, kLB | l0 <= k;
  // encoded r << 16 | k << 8 | l0 (-1 = none).  kSlots covers
  // kSrcRound * sum_k ceil((k + 1) / kLB) tasks.
  int task[kSlots];
  cx<R> sum[kSlots][kLB], comp[kSlots][kLB];
  int nb = 0;  // blocks per source
  for (int k = 0; k < p; ++k) nb += (k + kLB) / kLB;
#pragma unroll
  for (int j = 0; j < kSlots; ++j) {
    const int g = threadIdx.x + j * kThreads;
    task[j] = -1;
    if (g < kSrcRound * nb) {
      const int r = g / nb;
      int b = g - r * nb, k = 0;
      while (b >= (k + kLB) / kLB) b -= (k++ + kLB) / kLB;
      task[j] = (r << 16) | (k << 8) | (b * kLB);
    }
#pragma unroll
    for (int q = 0; q < kLB; ++q) sum[j][q] = comp[j][q] = {(R)0, (R)0};
  }
  for (int e = e0; e < e1; e += kSrcRound) {
    const int nr = min(kSrcRound, e1 - e);
    __syncthreads();
    // geometry and the per-degree factors, a thread per (source, degree)
    for (int g = threadIdx.x; g < nr * p; g += kThreads) {
      const int r = g / p, n = g - r * p;
      const int sa = src[e + r];
      R ux, uy, uz, rhoA, rhoB;
      if constexpr (sizeof(R) == 4) {
        const float dx = (float)(fc[3 * tb] - fc[3 * sa]), dy = (float)(fc[3 * tb + 1] - fc[3 * sa + 1]),
                    dz = (float)(fc[3 * tb + 2] - fc[3 * sa + 2]);
        const float inv = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
        ux = dx * inv;
        uy = dy * inv;
        uz = dz * inv;
        rhoA = ldexpf(inv, kMaxLevel - level[sa]);
        rhoB = ldexpf(inv, kMaxLevel - level[tb]);
      } else {
        const double dx = cen[3 * tb] - cen[3 * sa], dy = cen[3 * tb + 1] - cen[3 * sa + 1],
                     dz = cen[3 * tb + 2] - cen[3 * sa + 2];
        const double rr = sqrt(dx * dx + dy * dy + dz * dz);
        ux = dx / rr;
        uy = dy / rr;
        uz = dz / rr;
        rhoA = ldexp(root[9], -level[sa]) / rr;
        rhoB = ldexp(root[9], -level[tb]) / rr;
      }
      if (n == 0) {
        geo[3 * r] = ux;
        geo[3 * r + 1] = uy;
        geo[3 * r + 2] = uz;
      }
      R fa = 1, fb = rhoB;
      for (int q = 1; q <= n; ++q) {
        fa *= rhoA * (R)q;
        fb *= rhoB * (R)q;
      }
      gA[r * p + n] = fa;
      fk[r * p + n] = (n & 1) ? -fb : fb;
    }
    __syncthreads();
    // harmonics, a thread per (source, order column); scaled multipoles
    for (int g = threadIdx.x; g < nr * PT; g += kThreads) {
      const int r = g / PT, m = g - r * PT;
      irregular_column_full<R>(geo[3 * r], geo[3 * r + 1], geo[3 * r + 2], m, PT, rcp, T + r * nT);
    }
    for (int g = threadIdx.x; g < nr * nM; g += kThreads) {
      const int r = g / nM, i = g - r * nM;
      int n = (int)sqrtf((float)i);
      n -= n * n > i;
      const int m = i - n * n - n;  // -n .. n
      const int am = m < 0 ? -m : m;
      const R* mrow = M + (int64_t)src[e + r] * Kp;
      cx<R> v{mrow[ridx(n, am, 0)], am ? mrow[ridx(n, am, 1)] : (R)0};
      if (m < 0) {  // X_n^-m = (-1)^m conj(X_n^m)
        v.im = -v.im;
        if (am & 1) {
          v.re = -v.re;
          v.im = -v.im;
        }
      }
      const R f = gA[r * p + n];
      Mr[r * nM + i] = {v.re * f, v.im * f};
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kSlots; ++j) {
      const int tk = task[j];
      if (tk < 0 || (tk >> 16) >= nr) continue;
      const int r = tk >> 16, k = (tk >> 8) & 0xff, l0 = tk & 0xff;
      const cx<R>* Tr = T + r * nT;
      const cx<R>* Mq = Mr + r * nM;
      cx<R> acc[kLB];
#pragma unroll
      for (int q = 0; q < kLB; ++q) acc[q] = {(R)0, (R)0};
      for (int n = 0; n < p; ++n) {
        const int jd = n + k;
        // trow[m + q] = Th_{n+k}^{m+l0+q} / (n+k)!; past the row's end (l0 + q > k,
        // outputs that are not stored) it reads the next row or, for the last
        // row of the last slot, the first entries of Mr: inside the buffer.
        const cx<R>* trow = Tr + jd * jd + jd + l0;
        const cx<R>* mrow = Mq + n * n + n;  // mrow[m] = M~_n^m rho_A^n n!
        cx<R> an[kLB], win[kLB];
#pragma unroll
        for (int q = 0; q < kLB; ++q) an[q] = {(R)0, (R)0};
#pragma unroll
        for (int q = 0; q + 1 < kLB; ++q) win[q] = trow[-n + q];
#pragma unroll 4
        for (int m = -n; m <= n; ++m) {
          win[kLB - 1] = trow[m + kLB - 1];
          const cx<R> a = mrow[m];
#pragma unroll
          for (int q = 0; q < kLB; ++q) {
            an[q].re += a.re * win[q].re - a.im * win[q].im;
            an[q].im += a.re * win[q].im + a.im * win[q].re;
          }
#pragma unroll
          for (int q = 0; q + 1 < kLB; ++q) win[q] = win[q + 1];
        }
        const R b = bin[n * p + k];
#pragma unroll
        for (int q = 0; q < kLB; ++q) {
          acc[q].re += b * an[q].re;
          acc[q].im += b * an[q].im;
        }
      }
      const R f = fk[r * p + k];
#pragma unroll
      for (int q = 0; q < kLB; ++q) {
        {
          const R y = f * acc[q].re - comp[j][q].re, t = sum[j][q].re + y;
          comp[j][q].re = (t - sum[j][q].re) - y;
          sum[j][q].re = t;
        }
        {
          const R y = f * acc[q].im - comp[j][q].im, t = sum[j][q].im + y;
          comp[j][q].im = (t - sum[j][q].im) - y;
          sum[j][q].im = t;
        }
      }
    }
  }
  // slot sums in order (the harmonics buffer holds them: kSrcRound * nt <= kSrcRound * PT^2)
  __syncthreads();
  cx<R>* part = T;
#pragma unroll
  for (int j = 0; j < kSlots; ++j) {
    const int tk = task[j];
    if (tk < 0) continue;
    const int r = tk >> 16, k = (tk >> 8) & 0xff, l0 = tk & 0xff;
#pragma unroll
    for (int q = 0; q < kLB; ++q)
      if (l0 + q <= k) part[r * nt + tri(k, l0 + q)] = {sum[j][q].re - comp[j][q].re, sum[j][q].im - comp[j][q].im};
  }
  __syncthreads();
  R* out = L + (int64_t)tb * Kp;
  for (int o = threadIdx.x; o < nt; o += kThreads) {
    int k = 0;
    while ((k + 1) * (k + 2) / 2 <= o) ++k;
    const int l = o - k * (k + 1) / 2;
    cx<R> s{(R)0, (R)0};
    for (int r = 0; r < kSrcRound; ++r) {
      s.re += part[r * nt + o].re;
      s.im += part[r * nt + o].im;
    }
    out[ridx(k, l, 0)] = s.re;
    if (l) out[ridx(k, l, 1)] = s.im;
  }
}

// The sorted M2L list as CSR: ptr[c] = first pair with target >= c, and the
// targets that have sources.
__global__ void k_csr_ptr(const int32_t* __restrict__ tgt, int64_t n, int ncell, int32_t* __restrict__ ptr) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i > n) return;
  // pair i starts the targets in (tgt[i - 1], tgt[i]]
  const int lo = i == 0 ? 0 : tgt[i - 1] + 1;
  const int hi = i == n ? ncell : tgt[i];
  for (int c = lo; c <= hi && c <= ncell; ++c) ptr[c] = (int32_t)i;
}
__global__ void k_csr_targets(const int32_t* __restrict__ ptr, int ncell, int64_t* __restrict__ flag) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < ncell) flag[c] = ptr[c + 1] > ptr[c] ? 1 : 0;
}
__global__ void k_csr_compact(const int32_t* __restrict__ ptr, const int64_t* __restrict__ off, int ncell,
                              int32_t* __restrict__ tgts) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < ncell && ptr[c + 1] > ptr[c]) tgts[off[c]] = c;
}

}  // namespace

// Build-time state of the fitted far field: expansion centres and the M2L
// list by target (sorted by (target, source), so that each target adds its
// sources in a fixed order).
void build_fitted(fmm_tree* t) {
  Arena& a = t->arena;
  cudaStream_t s = t->stream;
  const int nc = t->ncell;
  t->fit_cen = alloc_n<double>(a, 3 * (size_t)nc);
  t->fit_cenf = alloc_n<float>(a, 6 * (size_t)nc);
  k_fit_centres<<<blocks(nc, 256), 256, 0, s>>>(t->fit_c, nc, t->d_root, t->fit_cen, t->fit_cenf);
  GB_LAUNCH("k_fit_centres");
  t->m2l_ptr = alloc_n<int32_t>(a, (size_t)nc + 1);
  t->m2l_csr_src = alloc_n<int32_t>(a, t->n_m2l);
  int32_t* tgt = alloc_n<int32_t>(a, t->n_m2l);
  sort_pairs_copy(a, t->m2l_tgt, t->m2l_src, t->n_m2l, nc, tgt, t->m2l_csr_src, s);
  k_csr_ptr<<<blocks(t->n_m2l + 1, 256), 256, 0, s>>>(tgt, t->n_m2l, nc, t->m2l_ptr);
  GB_LAUNCH("k_csr_ptr");
  int64_t* flag = alloc_n<int64_t>(a, nc);
  k_csr_targets<<<blocks(nc, 256), 256, 0, s>>>(t->m2l_ptr, nc, flag);
  GB_LAUNCH("k_csr_targets");
  t->fit_ntgt = (int)scan_exclusive_i64_total(a, flag, nc, s);
  t->fit_tgts = alloc_n<int32_t>(a, std::max(1, t->fit_ntgt));
  k_csr_compact<<<blocks(nc, 256), 256, 0, s>>>(t->m2l_ptr, flag, nc, t->fit_tgts);
  GB_LAUNCH("k_csr_compact");
  a.release(flag);
  a.release(tgt);
}

template <class R>
void launch_m2m_fit(fmm_tree* t, int level, cudaStream_t s) {
  const int first = t->level_begin[level], n = t->level_begin[level + 1] - first;
  if (n <= 0) return;
  k_m2m_fit<R><<<n, kThreads, 0, s>>>(first, n, t->c.cbeg, t->c.nch, t->c.level, t->fit_cen, t->d_root, t->p, t->Kp,
                                      (R*)t->M);
  GB_LAUNCH("k_m2m_fit");
}

template <class R>
void launch_l2l_fit(fmm_tree* t, int level, cudaStream_t s) {
  const int first = t->level_begin[level], n = t->level_begin[level + 1] - first;
  if (n <= 0) return;
  k_l2l_fit<R><<<n, kThreads, 0, s>>>(first, n, t->c.parent, t->c.level, t->fit_cen, t->d_root, t->p, t->Kp,
                                      (R*)t->L);
  GB_LAUNCH("k_l2l_fit");
}

template <class R>
void launch_m2l_fit(fmm_tree* t, cudaStream_t s) {
  if (t->fit_ntgt == 0) return;
  const int p = t->p, PT = 2 * p - 1;
  const size_t smem = sizeof(cx<R>) * (size_t)kSrcRound * (PT * PT + p * p) +
                      sizeof(R) * ((size_t)kSrcRound * (2 * p + 3) + p * p + 2 * kMaxP);
  // task slots per thread: kSrcRound * sum_k ceil((k + 1) / kLB) / kThreads
  // rounded up (96, 192 and 320 tasks at p = 8, 12, 16)
  auto kern = p <= 8 ? k_m2l_fit<R, 1> : p <= 12 ? k_m2l_fit<R, 2> : k_m2l_fit<R, 3>;
  GB_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<t->fit_ntgt, kThreads, smem, s>>>(t->m2l_ptr, t->fit_tgts, t->m2l_csr_src, t->c.level, t->fit_c, t->fit_cen,
                                           t->d_root, p, t->Kp, (const R*)t->M, (R*)t->L);
  GB_LAUNCH("k_m2l_fit");
}

template void launch_m2m_fit<float>(fmm_tree*, int, cudaStream_t);
template void launch_m2m_fit<double>(fmm_tree*, int, cudaStream_t);
template void launch_l2l_fit<float>(fmm_tree*, int, cudaStream_t);
template void launch_l2l_fit<double>(fmm_tree*, int, cudaStream_t);
template void launch_m2l_fit<float>(fmm_tree*, cudaStream_t);
template void launch_m2l_fit<double>(fmm_tree*, cudaStream_t);

}  // namespace gbfmm
