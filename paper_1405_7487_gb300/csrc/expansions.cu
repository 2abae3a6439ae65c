// expansions.cu -- P2M, M2M, L2L and L2P (Sec. II.A; Sec. II.C: P2M on the
// leaves and M2M on the other cells bottom up, L2L and L2P top down).
//
// Conventions (shared with the operator set-up in ops.cu):
//   M~_n^m(A) = sum_j q_j conj(Ups_n^m((y_j - c_A) / R_A))       (P2M)
//   phi(x)    = (1/R_B) sum_{k,l} L~_k^l conj(Ups_k^l((x - c_B) / R_B))   (L2P)
// with Ups_n^m the regular solid harmonics (Condon-Shortley phase),
// Ups_0^0 = 1, Ups_m^m = -(x + i y)/(2m) Ups_{m-1}^{m-1},
// (n+m)(n-m) Ups_n^m = (2n-1) z Ups_{n-1}^m - r^2 Ups_{n-2}^m,
// and the gradient from d/dz Ups_n^m = Ups_{n-1}^m,
// (d/dx +- i d/dy) Ups_n^m = +-Ups_{n-1}^{m+-1}.  Coefficients are stored
// for m >= 0 in the real packing n*n (+ 2m - 1, + 2m); the m < 0 half
// follows from X_n^{-m} = (-1)^m conj(X_n^m).
#include "kernels.cuh"

namespace gbfmm {
namespace {

constexpr int kWarps = 4;

__device__ __forceinline__ int ridx(int n, int m, int part) { return n * n + (m == 0 ? 0 : 2 * m - 1 + part); }

// Cell centre and half side in double: corner + (2k + 1) R, R = H 2^-level.
__device__ __forceinline__ void cell_geom(const double* __restrict__ root, int level, int ix, int iy, int iz,
                                          double c[3], double& R) {
  R = ldexp(root[9], -level);
  c[0] = root[10] + (2.0 * ix + 1.0) * R;
  c[1] = root[11] + (2.0 * iy + 1.0) * R;
  c[2] = root[12] + (2.0 * iz + 1.0) * R;
}

// The root cube as float pairs (corner hi + lo per axis, H hi + lo, 1/H),
// set up on the host from the double root box.
struct RootF {
  float ch[3], cl[3], hh, hl, ih;
};

// The frame of one cell for its bodies: the scaled offset (x - c) / R and
// 1/R.  The double path works in double.  The single path uses no FP64 (it
// runs at a small fraction of the FP32 rate): the centre c = corner +
// (2k + 1) R, R = H 2^-level, is formed as a float pair (an exact product
// by FMA and a compensated sum), and an offset is (x - c_hi) - c_lo in FP32
// -- x - c_hi is exact wherever the cell is at least its own size away from
// the origin, and small otherwise -- scaled by 1/R = 2^level / H in float.
// With particle-fitted centres (fcen / fcenf not null: 3 doubles, or hi[3]
// lo[3] floats, per cell) the centre is read instead; R stays the cube's half
// side.
template <class R>
struct Frame {
  double c[3], inv;
  __device__ void init(const double* __restrict__ root, const RootF&, int level, int ix, int iy, int iz, int cell,
                       const double* __restrict__ fcen, const float* __restrict__) {
    double Rc;
    cell_geom(root, level, ix, iy, iz, c, Rc);
    inv = 1.0 / Rc;
    if (fcen)
      for (int a = 0; a < 3; ++a) c[a] = fcen[3 * cell + a];
  }
  __device__ __forceinline__ R operator()(R x, int a) const { return (R)(((double)x - c[a]) * inv); }
  __device__ __forceinline__ R inv_r() const { return (R)inv; }
};
template <>
struct Frame<float> {
  float hi[3], lo[3], inv;
  __device__ void init(const double* __restrict__, const RootF& g, int level, int ix, int iy, int iz, int cell,
                       const double* __restrict__, const float* __restrict__ fcenf) {
    inv = ldexpf(g.ih, level);
    if (fcenf) {
      for (int a = 0; a < 3; ++a) {
        hi[a] = fcenf[6 * cell + a];
        lo[a] = fcenf[6 * cell + 3 + a];
      }
      return;
    }
    const float rh = ldexpf(g.hh, -level), rl = ldexpf(g.hl, -level);
    const int k3[3] = {ix, iy, iz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float k = (float)(2 * k3[a] + 1);  // < 2^22: exact
      const float p = k * rh;
      const float pe = fmaf(k, rh, -p) + k * rl;  // the product's low part
      const float s = g.ch[a] + p;
      const float bb = s - g.ch[a];
      const float se = (g.ch[a] - (s - bb)) + (p - bb);  // the sum's rounding error
      const float l = se + pe + g.cl[a];
      hi[a] = s + l;
      lo[a] = l - (hi[a] - s);
    }
  }
  __device__ __forceinline__ float operator()(float x, int a) const { return ((x - hi[a]) - lo[a]) * inv; }
  __device__ __forceinline__ float inv_r() const { return inv; }
};

template <class R, class R4>
__global__ void k_set_charges(const R4* __restrict__ bodies, const int32_t* __restrict__ perm,
                              const R* __restrict__ q, int64_t n, R4* __restrict__ work, Lim lim) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  R4 b = bodies[i];
  b.w = GB_LD(q, GB_LD(perm, i, lim.N, 301), lim.N, 302);
  work[i] = b;
}

// P2M: one warp per leaf.  The warp loads 32 bodies at a time (their scaled
// offsets from the centre, see Frame); the lanes form G = floor(32 / p)
// groups of p, lane m of a group owns column m of the expansion and runs the
// recurrence over n, and the groups take bodies in turn (G bodies per step).
// The groups' sums are added in group order at the end.
// Six blocks per SM (at most 80 registers a thread, a few spilled values).
template <class R, class R4>
__global__ void __launch_bounds__(32 * kWarps, 6) k_p2m(const R4* __restrict__ work, const int32_t* __restrict__ leaves, int nleaf,
                      const int32_t* __restrict__ level, const int32_t* __restrict__ ix,
                      const int32_t* __restrict__ iy, const int32_t* __restrict__ iz,
                      const int32_t* __restrict__ bbeg, const int32_t* __restrict__ bend,
                      const double* __restrict__ root, RootF rootf, const double* __restrict__ fcen,
                      const float* __restrict__ fcenf, int p, int Kp, R* __restrict__ M, Lim lim) {
  const int lane = threadIdx.x & 31;
  const int li = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (li >= nleaf) return;
  const int cell = leaves[li];
#ifdef GBFMM_CHECKED
  if (!in_range(cell, lim.ncell, 311, lim.rec)) return;
#endif
  Frame<R> off;
  off.init(root, rootf, level[cell], ix[cell], iy[cell], iz[cell], cell, fcen, fcenf);
  const int s = bbeg[cell], e = bend[cell];
  const int G = 32 / p;  // p <= 16: at least two groups
  const int g = lane / p, m = lane - g * p;
  const bool grp = g < G;
  R ar[kMaxP], ai[kMaxP], rf[kMaxP];
  // per-lane constants of column m: 1 / ((n+1+m)(n+1-m)) for n = m + k, and
  // the diagonal factor 1 / (2^m m!)
#pragma unroll
  for (int k = 0; k < kMaxP; ++k) {
    ar[k] = ai[k] = (R)0;
    rf[k] = (R)1 / ((R)(2 * m + k + 1) * (R)(k + 1));
  }
  R dfac = 1;
  for (int k = 1; k <= m; ++k) dfac /= (R)(2 * k);
  for (int j0 = s; j0 < e; j0 += 32) {
    R bx = 0, by = 0, bz = 0, bq = 0;
    if (j0 + lane < e) {
      R4 b = GB_LD(work, j0 + lane, lim.N, 312);
      bx = off(b.x, 0);
      by = off(b.y, 1);
      bz = off(b.z, 2);
      bq = b.w;
    }
    const int cnt = min(32, e - j0);
    // the trip count is warp-uniform: every lane takes part in every shuffle
    for (int jb = 0; jb < cnt; jb += G) {
      const int jj = jb + g;
      const bool ok = grp && jj < cnt;
      const int sl = ok ? jj : 0;
      const R x = __shfl_sync(0xffffffffu, bx, sl), y = __shfl_sync(0xffffffffu, by, sl);
      const R z = __shfl_sync(0xffffffffu, bz, sl), q = __shfl_sync(0xffffffffu, bq, sl);
      if (!ok) continue;
      // diagonal Ups_m^m = (-(x + i y))^m / (2^m m!)
      R ur = dfac, ui = 0;
      for (int k = 1; k <= m; ++k) {
        const R nr = -x * ur + y * ui;
        const R ni = -x * ui - y * ur;
        ur = nr;
        ui = ni;
      }
      const R r2 = x * x + y * y + z * z;
      R pr = 0, pi = 0;  // Ups_{n-2}^m
#pragma unroll
      for (int k = 0; k < kMaxP; ++k) {
        const int n = m + k;
        if (n < p) {
          // accumulate q conj(Ups_n^m)
          ar[k] += q * ur;
          ai[k] -= q * ui;
          // advance to n + 1
          const R f = rf[k];
          const R a = (R)(2 * n + 1) * z;
          const R nr = (a * ur - r2 * pr) * f;
          const R ni = (a * ui - r2 * pi) * f;
          pr = ur;
          pi = ui;
          ur = nr;
          ui = ni;
        }
      }
    }
  }
  // group 0 adds the other groups' sums in order (lane + j p < 32 for its lanes)
  for (int j = 1; j < G; ++j) {
    const int src = min(lane + j * p, 31);
#pragma unroll
    for (int k = 0; k < kMaxP; ++k) {
      const R vr = __shfl_sync(0xffffffffu, ar[k], src), vi = __shfl_sync(0xffffffffu, ai[k], src);
      if (g == 0) {
        ar[k] += vr;
        ai[k] += vi;
      }
    }
  }
  if (g == 0) {
    R* out = M + (int64_t)cell * Kp;
#pragma unroll
    for (int k = 0; k < kMaxP; ++k) {
      const int n = m + k;
      if (n < p) {
        GB_ST(out, ridx(n, m, 0), Kp, 313, ar[k]);
        if (m > 0) GB_ST(out, ridx(n, m, 1), Kp, 314, ai[k]);
      }
    }
  }
}

// M2M: one block per cell of a level; thread o forms output coefficient o
// from the children (operator matrices stored input-major per octant).
template <class R>
__global__ void k_m2m(int first, int ncell, const int32_t* __restrict__ cbeg, const int32_t* __restrict__ nch,
                      const int32_t* __restrict__ ix, const int32_t* __restrict__ iy,
                      const int32_t* __restrict__ iz, const R* __restrict__ opT, int K, int Kp,
                      R* __restrict__ M, Lim lim) {
  extern __shared__ unsigned char smem_raw[];
  R* Ms = reinterpret_cast<R*>(smem_raw);
  const int cell = first + blockIdx.x;
  if (blockIdx.x >= ncell) return;
  const int n = GB_LD(nch, cell, lim.ncell, 321);
  if (n == 0) return;
#ifdef GBFMM_CHECKED
  if (n > 8) {
    in_range(n, 9, 322, lim.rec);
    return;
  }
#endif
  const int c0 = cbeg[cell];
  for (int i = threadIdx.x; i < n * K; i += blockDim.x)
    Ms[i] = GB_LD(M, (int64_t)(c0 + i / K) * Kp + i % K, lim.ncell * lim.Kp, 323);
  __syncthreads();
  const int o = threadIdx.x;
  if (o >= K) return;
  R acc = 0;
  for (int c = 0; c < n; ++c) {
    const int ch = c0 + c;
    const int oct = ((GB_LD(ix, ch, lim.ncell, 324) & 1) << 2) | ((iy[ch] & 1) << 1) | (iz[ch] & 1);
    const R* op = opT + (int64_t)oct * Kp * Kp;
    const R* mc = Ms + c * K;
    for (int k = 0; k < K; ++k) acc += op[(int64_t)k * Kp + o] * mc[k];
  }
  GB_ST(M, (int64_t)cell * Kp + o, lim.ncell * lim.Kp, 325, acc);
}

// L2L: one block per cell of a level (>= 1): L(C) += op_oct(C) L(parent).
template <class R>
__global__ void k_l2l(int first, int ncell, const int32_t* __restrict__ parent,
                      const int32_t* __restrict__ ix, const int32_t* __restrict__ iy,
                      const int32_t* __restrict__ iz, const R* __restrict__ opT, int K, int Kp,
                      R* __restrict__ L, Lim lim) {
  extern __shared__ unsigned char smem_raw[];
  R* Ls = reinterpret_cast<R*>(smem_raw);
  const int cell = first + blockIdx.x;
  if (blockIdx.x >= ncell) return;
  const int par = GB_LD(parent, cell, lim.ncell, 331);
  for (int i = threadIdx.x; i < K; i += blockDim.x) Ls[i] = GB_LD(L, (int64_t)par * Kp + i, lim.ncell * lim.Kp, 332);
  __syncthreads();
  const int o = threadIdx.x;
  if (o >= K) return;
  const int oct = ((ix[cell] & 1) << 2) | ((iy[cell] & 1) << 1) | (iz[cell] & 1);
  const R* op = opT + (int64_t)oct * Kp * Kp;
  R acc = 0;
  for (int k = 0; k < K; ++k) acc += op[(int64_t)k * Kp + o] * Ls[k];
  GB_ST(L, (int64_t)cell * Kp + o, lim.ncell * lim.Kp, 333, L[(int64_t)cell * Kp + o] + acc);
}

// L2P and the output stage: one warp per leaf, lanes over its bodies.  The
// far field is added to the near field of P2P; forward mode writes the
// potential and force in input order and keeps (phi, grad) for the adjoint;
// backward mode forms dq = phi_w and dx = w grad phi_q + q grad phi_w.
template <class R, class R4>
__global__ void k_l2p_finalize(const R4* __restrict__ work, const int32_t* __restrict__ leaves, int nleaf,
                               const int32_t* __restrict__ level, const int32_t* __restrict__ ix,
                               const int32_t* __restrict__ iy, const int32_t* __restrict__ iz,
                               const int32_t* __restrict__ bbeg, const int32_t* __restrict__ bend,
                               const double* __restrict__ root, RootF rootf, const double* __restrict__ fcen,
                               const float* __restrict__ fcenf, int p, int Kp, const R* __restrict__ L,
                               const R4* __restrict__ near, const int32_t* __restrict__ perm, int mode,
                               R* __restrict__ out_a, R* __restrict__ out_b, R4* __restrict__ grad_q,
                               R* __restrict__ q_last, Lim lim) {
  extern __shared__ unsigned char smem_raw[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // reciprocal tables: rtab[m * kMaxP + n] = 1 / ((n+1+m)(n+1-m)), dtab[m] = 1 / (2m)
  R* rtab = reinterpret_cast<R*>(smem_raw);
  R* dtab = rtab + kMaxP * kMaxP;
  R* Ls = dtab + kMaxP + w * Kp;
  for (int i = threadIdx.x; i < kMaxP * kMaxP; i += blockDim.x) {
    const int mm = i / kMaxP, nn = i % kMaxP;
    rtab[i] = nn >= mm ? (R)1 / ((R)(nn + 1 + mm) * (R)(nn + 1 - mm)) : (R)0;
  }
  for (int i = threadIdx.x; i < kMaxP; i += blockDim.x) dtab[i] = i ? (R)1 / (R)(2 * i) : (R)0;
  __syncthreads();
  const int li = blockIdx.x * kWarps + w;
  if (li >= nleaf) return;
  const int cell = leaves[li];
#ifdef GBFMM_CHECKED
  if (!in_range(cell, lim.ncell, 341, lim.rec)) return;
#endif
  for (int i = lane; i < p * p; i += 32) Ls[i] = GB_LD(L, (int64_t)cell * Kp + i, lim.ncell * lim.Kp, 342);
  __syncwarp();
  Frame<R> off;
  off.init(root, rootf, level[cell], ix[cell], iy[cell], iz[cell], cell, fcen, fcenf);
  const R inv_r = off.inv_r();
  const int s = bbeg[cell], e = bend[cell];
  for (int i = s + lane; i < e; i += 32) {
    const R4 b = GB_LD(work, i, lim.N, 343);
    const R x = off(b.x, 0);
    const R y = off(b.y, 1);
    const R z = off(b.z, 2);
    const R r2 = x * x + y * y + z * z;
    R ph = 0, gx = 0, gy = 0, gz = 0;
    R dr = 1, di = 0;  // Ups_m^m
    for (int m = 0; m < p; ++m) {
      if (m > 0) {
        const R f = dtab[m];
        const R nr = (-x * dr + y * di) * f;
        const R ni = (-x * di - y * dr) * f;
        dr = nr;
        di = ni;
      }
      const R wm = m == 0 ? (R)1 : (R)2;
      R ur = dr, ui = di, pr = 0, pi = 0;
      // packed offsets of columns m, m - 1 and m + 1 within a degree (ridx),
      // the running n^2 and 2n + 1 (the latter also as a float)
      const int c0 = m ? 2 * m - 1 : 0, cm = m >= 2 ? 2 * m - 3 : 0, cp = 2 * m + 1;
      int sq = m * m, c = 2 * m + 1;
      R cf = (R)c;
      for (int n = m; n < p; ++n) {
        // Re(L conj U) = Lr Ur + Li Ui ; Im(L conj U) = Li Ur - Lr Ui
        {
          const R lr = Ls[sq + c0], lim = m ? Ls[sq + c0 + 1] : (R)0;
          ph += wm * (lr * ur + lim * ui);
        }
        const int sq1 = sq + c;  // (n + 1)^2
        if (n + 1 < p) {
          {
            const R lr = Ls[sq1 + c0], lim = m ? Ls[sq1 + c0 + 1] : (R)0;
            gz += wm * (lr * ur + lim * ui);
          }
          if (m >= 1) {
            const R lr = Ls[sq1 + cm], lim = (m - 1) ? Ls[sq1 + cm + 1] : (R)0;
            gx += lr * ur + lim * ui;
            gy -= lim * ur - lr * ui;
          }
          {
            const R lr = Ls[sq1 + cp], lim = Ls[sq1 + cp + 1];
            gx -= lr * ur + lim * ui;
            gy -= lim * ur - lr * ui;
          }
        }
        const R f = rtab[m * kMaxP + n];
        const R a = cf * z;
        const R nr = (a * ur - r2 * pr) * f;
        const R ni = (a * ui - r2 * pi) * f;
        pr = ur;
        pi = ui;
        ur = nr;
        ui = ni;
        sq = sq1;
        c += 2;
        cf += (R)2;
      }
    }
    const R4 nf = GB_LD(near, i, lim.N, 344);
    const R tphi = nf.x + ph * inv_r;
    const R i2 = inv_r * inv_r;
    const R tx = nf.y + gx * i2, ty = nf.z + gy * i2, tz = nf.w + gz * i2;
    const int64_t j = GB_LD(perm, i, lim.N, 345);
    if (mode == 0) {
      GB_ST(out_a, j, lim.N, 346, tphi);
      if (out_b) {
        GB_ST(out_b, 3 * j, 3 * lim.N, 347, -tx);
        GB_ST(out_b, 3 * j + 1, 3 * lim.N, 347, -ty);
        GB_ST(out_b, 3 * j + 2, 3 * lim.N, 347, -tz);
      }
      R4 g;
      g.x = tphi;
      g.y = tx;
      g.z = ty;
      g.w = tz;
      GB_ST(grad_q, i, lim.N, 348, g);
      GB_ST(q_last, i, lim.N, 349, b.w);
    } else {
      const R4 gq = GB_LD(grad_q, i, lim.N, 350);
      const R wq = b.w, qq = GB_LD(q_last, i, lim.N, 351);
      GB_ST(out_a, j, lim.N, 352, tphi);
      GB_ST(out_b, 3 * j, 3 * lim.N, 353, wq * gq.y + qq * tx);
      GB_ST(out_b, 3 * j + 1, 3 * lim.N, 353, wq * gq.z + qq * ty);
      GB_ST(out_b, 3 * j + 2, 3 * lim.N, 353, wq * gq.w + qq * tz);
    }
  }
}

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

namespace {
// The root cube's corner and half side as float pairs.
RootF root_f(const fmm_tree* t) {
  RootF g;
  for (int a = 0; a < 3; ++a) {
    g.ch[a] = (float)t->root.corner[a];
    g.cl[a] = (float)(t->root.corner[a] - (double)g.ch[a]);
  }
  g.hh = (float)t->root.H;
  g.hl = (float)(t->root.H - (double)g.hh);
  g.ih = (float)(1.0 / t->root.H);
  return g;
}
}  // namespace

template <class R>
void launch_set_charges(fmm_tree* t, const R* q, cudaStream_t s) {
  using R4 = typename Vec4<R>::type;
  k_set_charges<R, R4><<<blocks(t->N, 256), 256, 0, s>>>((const R4*)t->bodies, t->perm, q, t->N, (R4*)t->work, t->lim);
  GB_LAUNCH("k_set_charges");
}

template <class R>
void launch_p2m(fmm_tree* t, cudaStream_t s) {
  using R4 = typename Vec4<R>::type;
  k_p2m<R, R4><<<blocks(t->nleaf, kWarps), 32 * kWarps, 0, s>>>(
      (const R4*)t->work, t->leaves, t->nleaf, t->c.level, t->c.ix, t->c.iy, t->c.iz, t->c.bbeg, t->c.bend,
      t->d_root, root_f(t), t->fit_cen, t->fit_cenf, t->p, t->Kp, (R*)t->M, t->lim);
  GB_LAUNCH("k_p2m");
}

template <class R>
void launch_m2m(fmm_tree* t, int level, cudaStream_t s) {
  const int first = t->level_begin[level], n = t->level_begin[level + 1] - first;
  if (n <= 0) return;
  const int threads = ((t->K + 31) / 32) * 32;
  k_m2m<R><<<n, threads, sizeof(R) * 8 * t->K, s>>>(first, n, t->c.cbeg, t->c.nch, t->c.ix, t->c.iy, t->c.iz,
                                                    (const R*)t->m2m_ops, t->K, t->Kp, (R*)t->M, t->lim);
  GB_LAUNCH("k_m2m");
}

template <class R>
void launch_l2l(fmm_tree* t, int level, cudaStream_t s) {
  const int first = t->level_begin[level], n = t->level_begin[level + 1] - first;
  if (n <= 0) return;
  const int threads = ((t->K + 31) / 32) * 32;
  k_l2l<R><<<n, threads, sizeof(R) * t->K, s>>>(first, n, t->c.parent, t->c.ix, t->c.iy, t->c.iz,
                                                (const R*)t->l2l_ops, t->K, t->Kp, (R*)t->L, t->lim);
  GB_LAUNCH("k_l2l");
}

template <class R>
void launch_l2p_finalize(fmm_tree* t, int mode, R* a, R* b, cudaStream_t s) {
  using R4 = typename Vec4<R>::type;
  k_l2p_finalize<R, R4><<<blocks(t->nleaf, kWarps), 32 * kWarps,
                          sizeof(R) * (kMaxP * kMaxP + kMaxP + kWarps * t->Kp), s>>>(
      (const R4*)t->work, t->leaves, t->nleaf, t->c.level, t->c.ix, t->c.iy, t->c.iz, t->c.bbeg, t->c.bend,
      t->d_root, root_f(t), t->fit_cen, t->fit_cenf, t->p, t->Kp, (const R*)t->L, (const R4*)t->near, t->perm, mode,
      a, b, (R4*)t->grad_q, (R*)t->q_last, t->lim);
  GB_LAUNCH("k_l2p_finalize");
}

#define GB_INST(R)                                                         \
  template void launch_set_charges<R>(fmm_tree*, const R*, cudaStream_t);  \
  template void launch_p2m<R>(fmm_tree*, cudaStream_t);                    \
  template void launch_m2m<R>(fmm_tree*, int, cudaStream_t);               \
  template void launch_l2l<R>(fmm_tree*, int, cudaStream_t);               \
  template void launch_l2p_finalize<R>(fmm_tree*, int, R*, R*, cudaStream_t);
GB_INST(float)
GB_INST(double)
#undef GB_INST

}  // namespace gbfmm
