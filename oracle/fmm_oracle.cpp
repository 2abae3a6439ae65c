// fmm_oracle.cpp -- plain, slow, double-precision CPU reference of the FMM
// hot path (tree, dual tree traversal, P2M/M2M/M2L/L2L/L2P, P2P).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library or its
// Python binding) links, loads or calls this file.  Only the test-suite, the
// package smoke check and the CPU-baseline leg of the benchmark use it.  It
// shares no code, header, table or constant generator with the CUDA path.
//
// What it follows (AbdulJabbar, Yokota, Keyes, "Asynchronous Execution of the
// Fast Multipole Method Using Charm++"):
//   * Sec. II.A: the six FMM operators P2M, M2M, M2L, L2L, L2P, P2P, their
//     order (upward pass, M2L + P2P, downward pass), and the rule that a cell
//     may only take an M2L from a cell far enough compared with its size.
//   * Sec. II.B: Morton keys with three bits per level; a 64-bit key holds
//     21 levels.
//   * Sec. II.C: local tree from the bounding box; P2M on leaves, M2M on
//     non-leaves bottom up; M2L/P2P found by a dual tree traversal (Dehnen);
//     L2L/L2P top down.
//   * Sec. III.A / Table 1: P (order of expansion), theta (acceptance
//     criterion, error O(theta^P)), N_crit (maximum bodies per leaf).
// The paper leaves the expansion mathematics to Cheng et al.; the formulas
// below are the standard solid-harmonic ones, written out from the addition
// theorem, and each is pinned by the CPU tests (addition theorem, exact
// translation identities, an independent Cartesian Taylor checker, direct
// sums, invariants).
//
// Conventions (all readings of the paper are listed in the design notes):
//   * "order p" = p terms, degrees n = 0..p-1.
//   * Regular solid harmonics  Ups_n^m(r) = r^n P_n^m(cos t) e^{i m phi}/(n+m)!
//     Irregular                Th_n^m(r)  = (n-m)! P_n^m(cos t) e^{i m phi}/r^{n+1}
//     with the Condon-Shortley phase in P_n^m and  X_n^{-m} = (-1)^m conj(X_n^m).
//     1/|x-y| = sum_{n,m} conj(Ups_n^m(y)) Th_n^m(x)           (|y| < |x|)
//   * P2M  M_n^m(A) = sum_j q_j conj(Ups_n^m(y_j - c_A))
//     M2M  M_n^m(P) = sum_{k,l} M_k^l(C) conj(Ups_{n-k}^{m-l}(c_C - c_P))
//     M2L  L_k^l(B) = (-1)^k sum_{n,m} M_n^m(A) Th_{n+k}^{m+l}(c_B - c_A)
//     L2L  L_j^i(C) = sum_{k,l} L_k^l(P) conj(Ups_{k-j}^{l-i}(c_C - c_P))
//     L2P  phi(x)   = sum_{k,l} L_k^l conj(Ups_k^l(x - c_B))
//     gradient from  d/dz Ups_n^m = Ups_{n-1}^m,
//                    (d/dx + i d/dy) Ups_n^m =  Ups_{n-1}^{m+1},
//                    (d/dx - i d/dy) Ups_n^m = -Ups_{n-1}^{m-1}.
//   * Expansions are stored as full complex arrays, index n*(n+1)+m for
//     -n <= m <= n (p*p entries); no m >= 0 symmetry is used here.
//   * Output: phi_i (no 1/(4 pi), no softening), grad_i = grad phi(x_i);
//     self and coincident pairs contribute zero.
//   * Range: the harmonics are unscaled (r^n and 1/r^(n+1) up to degree
//     2p - 2), so the far field needs those powers of the cell sizes and
//     distances inside the double range: at p = 16 a root cube between about
//     1e-9 and 1e9 across.  The tree, the lists and the near field have no
//     such limit.
//
// Build:  g++ -O2 -std=c++17 -fopenmp -ffp-contract=off -fPIC -shared

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef std::complex<double> cplx;

namespace {

const int MAXLEVEL = 21;  // 63-bit Morton key, 3 bits per level (Sec. II.B)

inline int hidx(int n, int m) { return n * (n + 1) + m; }

// Regular solid harmonics Ups_n^m(v) for 0 <= n < P, -n <= m <= n.
// Recurrences: Ups_0^0 = 1, Ups_m^m = -(x+iy)/(2m) Ups_{m-1}^{m-1},
// (n+m)(n-m) Ups_n^m = (2n-1) z Ups_{n-1}^m - r^2 Ups_{n-2}^m.
void regular(const double v[3], int P, cplx* U) {
  const double x = v[0], y = v[1], z = v[2];
  const double r2 = x * x + y * y + z * z;
  const cplx xy(x, y);
  if (P <= 0) return;
  U[hidx(0, 0)] = 1.0;
  for (int m = 1; m < P; ++m) U[hidx(m, m)] = U[hidx(m - 1, m - 1)] * (-xy) / (2.0 * m);
  for (int m = 0; m < P; ++m) {
    for (int n = m + 1; n < P; ++n) {
      cplx a = U[hidx(n - 1, m)];
      cplx b = (n - 2 >= m) ? U[hidx(n - 2, m)] : cplx(0.0);
      U[hidx(n, m)] = ((2.0 * n - 1.0) * z * a - r2 * b) / double((n + m) * (n - m));
    }
  }
  for (int n = 1; n < P; ++n)
    for (int m = 1; m <= n; ++m)
      U[hidx(n, -m)] = ((m & 1) ? -1.0 : 1.0) * std::conj(U[hidx(n, m)]);
}

// Irregular solid harmonics Th_n^m(v) for 0 <= n < P.
// Th_0^0 = 1/r, Th_m^m = -(2m-1)(x+iy)/r^2 Th_{m-1}^{m-1},
// Th_n^m = ((2n-1) z Th_{n-1}^m - (n+m-1)(n-m-1) Th_{n-2}^m) / r^2.
void irregular(const double v[3], int P, cplx* T) {
  const double x = v[0], y = v[1], z = v[2];
  const double r2 = x * x + y * y + z * z;
  const cplx xy(x, y);
  if (P <= 0) return;
  T[hidx(0, 0)] = 1.0 / std::sqrt(r2);
  for (int m = 1; m < P; ++m)
    T[hidx(m, m)] = T[hidx(m - 1, m - 1)] * (-(2.0 * m - 1.0)) * xy / r2;
  for (int m = 0; m < P; ++m) {
    for (int n = m + 1; n < P; ++n) {
      cplx a = T[hidx(n - 1, m)];
      cplx b = (n - 2 >= m) ? T[hidx(n - 2, m)] : cplx(0.0);
      T[hidx(n, m)] = ((2.0 * n - 1.0) * z * a - double((n + m - 1) * (n - m - 1)) * b) / r2;
    }
  }
  for (int n = 1; n < P; ++n)
    for (int m = 1; m <= n; ++m)
      T[hidx(n, -m)] = ((m & 1) ? -1.0 : 1.0) * std::conj(T[hidx(n, m)]);
}

// ---------------------------------------------------------------- operators
// All operate on full complex coefficient arrays of p*p entries.

// P2M: M += sum_j q_j conj(Ups(y_j - c))
void op_p2m(int p, const double c[3], int nb, const double* xyz, const double* q, cplx* M) {
  std::vector<cplx> U(p * p);
  for (int j = 0; j < nb; ++j) {
    double v[3] = {xyz[3 * j] - c[0], xyz[3 * j + 1] - c[1], xyz[3 * j + 2] - c[2]};
    regular(v, p, U.data());
    for (int i = 0; i < p * p; ++i) M[i] += q[j] * std::conj(U[i]);
  }
}

// M2M: Mp += translate(Mc) from child centre cc to parent centre cp
void op_m2m(int p, const cplx* Mc, const double cc[3], const double cp[3], cplx* Mp) {
  std::vector<cplx> U(p * p);
  double t[3] = {cc[0] - cp[0], cc[1] - cp[1], cc[2] - cp[2]};
  regular(t, p, U.data());
  for (int n = 0; n < p; ++n)
    for (int m = -n; m <= n; ++m) {
      cplx s = 0.0;
      for (int k = 0; k <= n; ++k)
        for (int l = -k; l <= k; ++l) {
          int dm = m - l;
          if (dm < -(n - k) || dm > (n - k)) continue;
          s += Mc[hidx(k, l)] * std::conj(U[hidx(n - k, dm)]);
        }
      Mp[hidx(n, m)] += s;
    }
}

// M2L: L(B) += conversion of M(A); d = c_B - c_A
void op_m2l(int p, const cplx* M, const double cA[3], const double cB[3], cplx* L) {
  const int PT = 2 * p - 1;
  std::vector<cplx> T(PT * PT);
  double d[3] = {cB[0] - cA[0], cB[1] - cA[1], cB[2] - cA[2]};
  irregular(d, PT, T.data());
  for (int k = 0; k < p; ++k)
    for (int l = -k; l <= k; ++l) {
      cplx s = 0.0;
      for (int n = 0; n < p; ++n)
        for (int m = -n; m <= n; ++m)
          s += M[hidx(n, m)] * T[hidx(n + k, m + l)];
      L[hidx(k, l)] += ((k & 1) ? -1.0 : 1.0) * s;
    }
}

// L2L: Lc += shift of Lp from parent centre cp to child centre cc
void op_l2l(int p, const cplx* Lp, const double cp[3], const double cc[3], cplx* Lc) {
  std::vector<cplx> U(p * p);
  double t[3] = {cc[0] - cp[0], cc[1] - cp[1], cc[2] - cp[2]};
  regular(t, p, U.data());
  for (int j = 0; j < p; ++j)
    for (int i = -j; i <= j; ++i) {
      cplx s = 0.0;
      for (int k = j; k < p; ++k)
        for (int l = -k; l <= k; ++l) {
          int dl = l - i;
          if (dl < -(k - j) || dl > (k - j)) continue;
          s += Lp[hidx(k, l)] * std::conj(U[hidx(k - j, dl)]);
        }
      Lc[hidx(j, i)] += s;
    }
}

// L2P: potential and gradient of the local expansion L about c at point x.
void op_l2p(int p, const cplx* L, const double c[3], const double x[3], double* phi, double g[3]) {
  std::vector<cplx> U(p * p);
  double v[3] = {x[0] - c[0], x[1] - c[1], x[2] - c[2]};
  regular(v, p, U.data());
  cplx sphi = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
  for (int k = 0; k < p; ++k)
    for (int l = -k; l <= k; ++l) {
      const cplx Lk = L[hidx(k, l)];
      sphi += Lk * std::conj(U[hidx(k, l)]);
      if (k == 0) continue;
      // derivatives of Ups_k^l, each a degree k-1 harmonic (zero if |m| > k-1)
      cplx up = (std::abs(l + 1) <= k - 1) ? U[hidx(k - 1, l + 1)] : cplx(0.0);
      cplx um = (std::abs(l - 1) <= k - 1) ? U[hidx(k - 1, l - 1)] : cplx(0.0);
      cplx uz = (std::abs(l) <= k - 1) ? U[hidx(k - 1, l)] : cplx(0.0);
      // d+ = up, d- = -um;  dx = (d+ + d-)/2, dy = (d+ - d-)/(2i)
      cplx dxU = 0.5 * (up - um);
      cplx dyU = (up + um) / cplx(0.0, 2.0);
      sx += Lk * std::conj(dxU);
      sy += Lk * std::conj(dyU);
      sz += Lk * std::conj(uz);
    }
  *phi += sphi.real();
  g[0] += sx.real();
  g[1] += sy.real();
  g[2] += sz.real();
}

// M2P: potential and gradient of a multipole expansion M about c at x
// (used only by the pins: it evaluates sum M_n^m Th_n^m(x - c)).
void op_m2p(int p, const cplx* M, const double c[3], const double x[3], double* phi, double g[3]) {
  // gradient from the ladder relations of the irregular harmonics:
  // d/dz Th_n^m = -Th_{n+1}^m, (d/dx + i d/dy) Th_n^m = Th_{n+1}^{m+1},
  // (d/dx - i d/dy) Th_n^m = -Th_{n+1}^{m-1}.
  const int PT = p + 1;
  std::vector<cplx> T(PT * PT);
  double v[3] = {x[0] - c[0], x[1] - c[1], x[2] - c[2]};
  irregular(v, PT, T.data());
  cplx sphi = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
  for (int n = 0; n < p; ++n)
    for (int m = -n; m <= n; ++m) {
      const cplx Mn = M[hidx(n, m)];
      sphi += Mn * T[hidx(n, m)];
      cplx dp = T[hidx(n + 1, m + 1)];
      cplx dm = -T[hidx(n + 1, m - 1)];
      sx += Mn * 0.5 * (dp + dm);
      sy += Mn * (dp - dm) / cplx(0.0, 2.0);
      sz += Mn * (-T[hidx(n + 1, m)]);
    }
  *phi += sphi.real();
  g[0] += sx.real();
  g[1] += sy.real();
  g[2] += sz.real();
}

}  // namespace

// ------------------------------------------------------------------- tree
namespace {

struct Tree {
  int64_t N = 0;
  int p = 0;
  double theta = 0;
  int ncrit = 0;
  int circumscribed = 0;
  int tight = 0;                         // particle-fitted MAC radius (Sec. II.B)
  int fitted = 0;                        // expansion centres at the particle-fitted box (Sec. II.B)
  std::vector<int64_t> r2;               // squared radius per cell (tight or fitted)
  std::vector<int64_t> cint;             // fitted: 3 integer centre coordinates per cell (units H / 2^21)
  double lo[3], hi[3], ctr[3], H = 0, r0[3];
  std::vector<double> xyz, q;            // input order (3N, N)
  std::vector<uint64_t> key_sorted;      // keys in sorted order
  std::vector<int64_t> perm;             // sorted position -> input index
  std::vector<int> level, ix, iy, iz, bbeg, bend, cbeg, nch, parent;
  std::vector<int> level_begin;          // first cell of each level (+ end)
  std::vector<int> p2p_src, p2p_tgt, m2l_src, m2l_tgt;  // sorted by (tgt, src)
  std::vector<int64_t> p2p_ptr, m2l_ptr; // CSR by target cell
  std::vector<cplx> M, L;                // last evaluation, cells x p*p
};

// Spread the low 21 bits of v so that bit b goes to bit 3b.
uint64_t spread3(uint64_t v) {
  uint64_t r = 0;
  for (int b = 0; b < MAXLEVEL; ++b) r |= ((v >> b) & 1ull) << (3 * b);
  return r;
}
uint64_t gather3(uint64_t k) {
  uint64_t r = 0;
  for (int b = 0; b < MAXLEVEL; ++b) r |= ((k >> (3 * b)) & 1ull) << b;
  return r;
}

// Root cube and per-body integer coordinates (Sec. II.B, II.C: keys from the
// local bounding box).  Evaluated in IEEE double in exactly this order; the
// build flags forbid contraction into fused multiply-adds.
void root_and_keys(Tree& t, std::vector<uint64_t>& key_in) {
  const int64_t N = t.N;
  for (int a = 0; a < 3; ++a) {
    double lo = t.xyz[a], hi = t.xyz[a];
    for (int64_t i = 1; i < N; ++i) {
      double v = t.xyz[3 * i + a];
      lo = std::min(lo, v);
      hi = std::max(hi, v);
    }
    t.lo[a] = lo;
    t.hi[a] = hi;
    t.ctr[a] = (lo + hi) * 0.5;
  }
  double h = 0.0;
  for (int a = 0; a < 3; ++a) h = std::max(h, (t.hi[a] - t.lo[a]) * 0.5);
  t.H = h * (1.0 + std::ldexp(1.0, -20));
  if (t.H == 0.0) t.H = 0.5;
  for (int a = 0; a < 3; ++a) t.r0[a] = t.ctr[a] - t.H;
  // voxels per unit length, 2^21 / (2H), rounded once
  const double per_len = std::ldexp(1.0, MAXLEVEL) / (2.0 * t.H);
  const int64_t kmax = (1ll << MAXLEVEL) - 1;
  key_in.resize(N);
  for (int64_t i = 0; i < N; ++i) {
    uint64_t k3[3];
    for (int a = 0; a < 3; ++a) {
      double d = t.xyz[3 * i + a] - t.r0[a];
      double s = d * per_len;
      double fl = std::floor(s);
      int64_t k = (int64_t)fl;
      if (k < 0) k = 0;
      if (k > kmax) k = kmax;
      k3[a] = (uint64_t)k;
    }
    key_in[i] = (spread3(k3[0]) << 2) | (spread3(k3[1]) << 1) | spread3(k3[2]);
  }
}

// Level-wise construction: a cell at level l over bodies [s, e) is split iff
// e - s > ncrit and l < 21 (Sec. III.A: N_crit is the maximum number of bodies
// per leaf); children are the nonempty octants in Morton order.  Cells are
// numbered breadth first, i.e. by (level, Morton key).
void build_cells(Tree& t) {
  const int64_t N = t.N;
  auto add_cell = [&](int l, int s, int e, int par) {
    uint64_t k = t.key_sorted[s];
    int shift = MAXLEVEL - l;
    t.level.push_back(l);
    t.ix.push_back((int)(gather3(k >> 2) >> shift));
    t.iy.push_back((int)(gather3(k >> 1) >> shift));
    t.iz.push_back((int)(gather3(k) >> shift));
    t.bbeg.push_back(s);
    t.bend.push_back(e);
    t.cbeg.push_back(-1);
    t.nch.push_back(0);
    t.parent.push_back(par);
  };
  add_cell(0, 0, (int)N, -1);
  t.level_begin.push_back(0);
  int lbeg = 0, lend = 1;
  for (int l = 0; l < MAXLEVEL && lbeg < lend; ++l) {
    t.level_begin.push_back(lend);
    for (int c = lbeg; c < lend; ++c) {
      int s = t.bbeg[c], e = t.bend[c];
      if (e - s <= t.ncrit) continue;
      int first = (int)t.level.size();
      int shift = 3 * (MAXLEVEL - l - 1);
      int i = s;
      while (i < e) {
        uint64_t oct = (t.key_sorted[i] >> shift) & 7ull;
        int j = i;
        while (j < e && ((t.key_sorted[j] >> shift) & 7ull) == oct) ++j;
        add_cell(l + 1, i, j, c);
        i = j;
      }
      t.cbeg[c] = first;
      t.nch[c] = (int)t.level.size() - first;
    }
    lbeg = lend;
    lend = (int)t.level.size();
  }
  if (t.level_begin.back() != (int)t.level.size()) t.level_begin.push_back((int)t.level.size());
  // drop empty trailing levels
  while (t.level_begin.size() >= 2 &&
         t.level_begin[t.level_begin.size() - 1] == t.level_begin[t.level_begin.size() - 2])
    t.level_begin.pop_back();
}

// Multipole acceptance criterion, theta * |c_A - c_B| > R_A + R_B, evaluated
// on exact integers: centres are (2k+1) 2^(21-l) and radii 2^(21-l) in units
// of H / 2^21 (R = half side; the circumscribed radius multiplies by sqrt 3).
//
// Particle-fitted variant (tight): the radius of a cell is the distance from
// its centre to its farthest body, in the same units, each body at the centre
// 2u + 1 of its voxel u (its 21-bit integer coordinate).  The squared radius
// is an exact integer; the test is theta^2 D^2 > (sqrt(r2_A) + sqrt(r2_B))^2
// in IEEE double (square roots correctly rounded, no contraction).
void tight_radii(Tree& t) {
  const int n = (int)t.level.size();
  t.r2.assign(n, 0);
  for (int c = 0; c < n; ++c) {
    const int sh = MAXLEVEL - t.level[c];
    const int64_t ctr[3] = {(2ll * t.ix[c] + 1) << sh, (2ll * t.iy[c] + 1) << sh, (2ll * t.iz[c] + 1) << sh};
    int64_t best = 0;
    for (int i = t.bbeg[c]; i < t.bend[c]; ++i) {
      const uint64_t k = t.key_sorted[i];
      const int64_t u[3] = {(int64_t)gather3(k >> 2), (int64_t)gather3(k >> 1), (int64_t)gather3(k)};
      int64_t d2 = 0;
      for (int a = 0; a < 3; ++a) {
        const int64_t d = 2 * u[a] + 1 - ctr[a];
        d2 += d * d;
      }
      best = std::max(best, d2);
    }
    t.r2[c] = best;
  }
}

// Particle-fitted centres (fitted): per axis the box of the cell's voxel
// centres 2u + 1 runs from 2 u_min + 1 to 2 u_max + 1, so its centre is the
// integer u_min + u_max + 1 (units of H / 2^21); the radius is the distance
// from that centre to the farthest voxel centre, its square an exact integer.
// The MAC then measures |c_A - c_B| between the fitted centres, and every
// expansion (P2M, M2M, M2L, L2L, L2P) is taken about them.
void fitted_centres(Tree& t) {
  const int n = (int)t.level.size();
  t.r2.assign(n, 0);
  t.cint.assign(3 * (size_t)n, 0);
  for (int c = 0; c < n; ++c) {
    int64_t lo[3] = {INT64_MAX, INT64_MAX, INT64_MAX}, hi[3] = {-1, -1, -1};
    for (int i = t.bbeg[c]; i < t.bend[c]; ++i) {
      const uint64_t k = t.key_sorted[i];
      const int64_t u[3] = {(int64_t)gather3(k >> 2), (int64_t)gather3(k >> 1), (int64_t)gather3(k)};
      for (int a = 0; a < 3; ++a) {
        lo[a] = std::min(lo[a], u[a]);
        hi[a] = std::max(hi[a], u[a]);
      }
    }
    int64_t ctr[3];
    for (int a = 0; a < 3; ++a) ctr[a] = t.cint[3 * (size_t)c + a] = lo[a] + hi[a] + 1;
    int64_t best = 0;
    for (int i = t.bbeg[c]; i < t.bend[c]; ++i) {
      const uint64_t k = t.key_sorted[i];
      const int64_t u[3] = {(int64_t)gather3(k >> 2), (int64_t)gather3(k >> 1), (int64_t)gather3(k)};
      int64_t d2 = 0;
      for (int a = 0; a < 3; ++a) {
        const int64_t d = 2 * u[a] + 1 - ctr[a];
        d2 += d * d;
      }
      best = std::max(best, d2);
    }
    t.r2[c] = best;
  }
}

bool mac(const Tree& t, int A, int B) {
  const int la = t.level[A], lb = t.level[B];
  int64_t dx = ((2ll * t.ix[A] + 1) << (MAXLEVEL - la)) - ((2ll * t.ix[B] + 1) << (MAXLEVEL - lb));
  int64_t dy = ((2ll * t.iy[A] + 1) << (MAXLEVEL - la)) - ((2ll * t.iy[B] + 1) << (MAXLEVEL - lb));
  int64_t dz = ((2ll * t.iz[A] + 1) << (MAXLEVEL - la)) - ((2ll * t.iz[B] + 1) << (MAXLEVEL - lb));
  if (t.fitted) {
    dx = t.cint[3 * (size_t)A] - t.cint[3 * (size_t)B];
    dy = t.cint[3 * (size_t)A + 1] - t.cint[3 * (size_t)B + 1];
    dz = t.cint[3 * (size_t)A + 2] - t.cint[3 * (size_t)B + 2];
  }
  int64_t D2 = dx * dx + dy * dy + dz * dz;
  if (t.tight || t.fitted) {
    const double sr = std::sqrt((double)t.r2[A]) + std::sqrt((double)t.r2[B]);
    return (t.theta * t.theta) * (double)D2 > sr * sr;
  }
  int64_t rs = (1ll << (MAXLEVEL - la)) + (1ll << (MAXLEVEL - lb));
  int64_t S2 = rs * rs;
  if (t.circumscribed) S2 *= 3;
  return (t.theta * t.theta) * (double)D2 > (double)S2;
}

// Dual tree traversal over unordered cell pairs, started from {root, root}
// (Sec. II.C, after Dehnen).  Rules:
//   {A,A}: a leaf interacts with itself by P2P; otherwise every unordered
//          pair of its children is visited.
//   {A,B}: accepted by the MAC -> M2L both ways; two leaves -> P2P both ways;
//          otherwise split the larger cell (the smaller level), or, if the
//          larger one is a leaf, the other one; equal sizes and both split-
//          table -> every pair (child of A, child of B).
// Lists are recorded as directed (source, target) pairs.
struct Traversal {
  const Tree& t;
  std::vector<std::pair<int, int>> p2p, m2l;  // (target, source)
  explicit Traversal(const Tree& tt) : t(tt) {}
  bool leaf(int c) const { return t.nch[c] == 0; }
  void visit(int A, int B) {
    if (A == B) {
      if (leaf(A)) {
        p2p.push_back({A, A});
        return;
      }
      for (int i = 0; i < t.nch[A]; ++i)
        for (int j = i; j < t.nch[A]; ++j) visit(t.cbeg[A] + i, t.cbeg[A] + j);
      return;
    }
    if (mac(t, A, B)) {
      m2l.push_back({B, A});
      m2l.push_back({A, B});
      return;
    }
    const bool la = leaf(A), lb = leaf(B);
    if (la && lb) {
      p2p.push_back({B, A});
      p2p.push_back({A, B});
      return;
    }
    int split;  // 0: A, 1: B, 2: both
    if (t.level[A] < t.level[B]) split = la ? 1 : 0;
    else if (t.level[B] < t.level[A]) split = lb ? 0 : 1;
    else split = (!la && !lb) ? 2 : (la ? 1 : 0);
    if (split == 2) {
      for (int i = 0; i < t.nch[A]; ++i)
        for (int j = 0; j < t.nch[B]; ++j) visit(t.cbeg[A] + i, t.cbeg[B] + j);
    } else if (split == 0) {
      for (int i = 0; i < t.nch[A]; ++i) visit(t.cbeg[A] + i, B);
    } else {
      for (int j = 0; j < t.nch[B]; ++j) visit(A, t.cbeg[B] + j);
    }
  }
};

void make_csr(int ncell, std::vector<std::pair<int, int>>& pairs, std::vector<int>& src,
              std::vector<int>& tgt, std::vector<int64_t>& ptr) {
  std::sort(pairs.begin(), pairs.end());
  src.resize(pairs.size());
  tgt.resize(pairs.size());
  ptr.assign(ncell + 1, 0);
  for (size_t i = 0; i < pairs.size(); ++i) {
    tgt[i] = pairs[i].first;
    src[i] = pairs[i].second;
    ptr[pairs[i].first + 1]++;
  }
  for (int c = 0; c < ncell; ++c) ptr[c + 1] += ptr[c];
}

void cell_centre(const Tree& t, int c, double out[3]) {
  if (t.fitted) {
    const double unit = std::ldexp(t.H, -MAXLEVEL);
    for (int a = 0; a < 3; ++a) out[a] = t.r0[a] + (double)t.cint[3 * (size_t)c + a] * unit;
    return;
  }
  const double R = std::ldexp(t.H, -t.level[c]);
  out[0] = t.r0[0] + (2.0 * t.ix[c] + 1.0) * R;
  out[1] = t.r0[1] + (2.0 * t.iy[c] + 1.0) * R;
  out[2] = t.r0[2] + (2.0 * t.iz[c] + 1.0) * R;
}

// Evaluation.  mode bit 1: near field (P2P), bit 2: far field (L2P).
// xyz_in: positions in input order (the build's unless overridden: the tree,
// lists and centres stay frozen).  targets: sorted positions to evaluate, or
// all when null.
void evaluate(Tree& t, const double* xyz_in, const double* q_in, int mode, int64_t ntarget,
              const int64_t* target_sorted, double* phi_s, double* grad_s) {
  const int p = t.p, K = p * p;
  const int ncell = (int)t.level.size();
  const int64_t N = t.N;
  std::vector<double> xs(3 * N), qs(N);
  for (int64_t i = 0; i < N; ++i) {
    int64_t j = t.perm[i];
    xs[3 * i] = xyz_in[3 * j];
    xs[3 * i + 1] = xyz_in[3 * j + 1];
    xs[3 * i + 2] = xyz_in[3 * j + 2];
    qs[i] = q_in[j];
  }
  std::vector<double> cen(3 * ncell);
  for (int c = 0; c < ncell; ++c) cell_centre(t, c, &cen[3 * c]);
  t.M.assign((size_t)ncell * K, cplx(0.0));
  t.L.assign((size_t)ncell * K, cplx(0.0));
  // Which cells need a local expansion: every cell when all targets are
  // wanted, else the ancestors of the wanted bodies' leaves.
  std::vector<int> leaf_of(N, -1);
  for (int c = 0; c < ncell; ++c)
    if (t.nch[c] == 0)
      for (int i = t.bbeg[c]; i < t.bend[c]; ++i) leaf_of[i] = c;
  std::vector<char> need(ncell, target_sorted ? 0 : 1);
  if (target_sorted)
    for (int64_t k = 0; k < ntarget; ++k)
      for (int c = leaf_of[target_sorted[k]]; c >= 0 && !need[c]; c = t.parent[c]) need[c] = 1;
  const int nlev = (int)t.level_begin.size() - 1;
  if (mode & 2) {
    // upward pass: P2M on leaves, M2M bottom up (Sec. II.C)
#pragma omp parallel for schedule(dynamic, 16)
    for (int c = 0; c < ncell; ++c)
      if (t.nch[c] == 0)
        op_p2m(p, &cen[3 * c], t.bend[c] - t.bbeg[c], &xs[3 * t.bbeg[c]], &qs[t.bbeg[c]],
               &t.M[(size_t)c * K]);
    for (int l = nlev - 1; l >= 0; --l) {
#pragma omp parallel for schedule(dynamic, 16)
      for (int c = t.level_begin[l]; c < t.level_begin[l + 1]; ++c)
        for (int i = 0; i < t.nch[c]; ++i) {
          int ch = t.cbeg[c] + i;
          op_m2m(p, &t.M[(size_t)ch * K], &cen[3 * ch], &cen[3 * c], &t.M[(size_t)c * K]);
        }
    }
    // M2L over the lists
#pragma omp parallel for schedule(dynamic, 4)
    for (int c = 0; c < ncell; ++c) {
      if (!need[c]) continue;
      for (int64_t e = t.m2l_ptr[c]; e < t.m2l_ptr[c + 1]; ++e) {
        int a = t.m2l_src[e];
        op_m2l(p, &t.M[(size_t)a * K], &cen[3 * a], &cen[3 * c], &t.L[(size_t)c * K]);
      }
    }
    // downward pass: L2L top down
    for (int l = 1; l < nlev; ++l) {
#pragma omp parallel for schedule(dynamic, 16)
      for (int c = t.level_begin[l]; c < t.level_begin[l + 1]; ++c) {
        if (!need[c]) continue;
        int par = t.parent[c];
        op_l2l(p, &t.L[(size_t)par * K], &cen[3 * par], &cen[3 * c], &t.L[(size_t)c * K]);
      }
    }
  }
  const int64_t nt = target_sorted ? ntarget : N;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t k = 0; k < nt; ++k) {
    const int64_t i = target_sorted ? target_sorted[k] : k;
    const int c = leaf_of[i];
    const double* xi = &xs[3 * i];
    double ph = 0.0, g[3] = {0.0, 0.0, 0.0};
    if (mode & 2) op_l2p(p, &t.L[(size_t)c * K], &cen[3 * c], xi, &ph, g);
    if (mode & 1) {
      for (int64_t e = t.p2p_ptr[c]; e < t.p2p_ptr[c + 1]; ++e) {
        int a = t.p2p_src[e];
        for (int j = t.bbeg[a]; j < t.bend[a]; ++j) {
          double dx = xi[0] - xs[3 * j], dy = xi[1] - xs[3 * j + 1], dz = xi[2] - xs[3 * j + 2];
          double r2 = dx * dx + dy * dy + dz * dz;
          if (r2 == 0.0) continue;  // self and coincident bodies
          double inv = 1.0 / std::sqrt(r2);
          double qi = qs[j] * inv;
          ph += qi;
          double f = qi * inv * inv;
          g[0] -= f * dx;
          g[1] -= f * dy;
          g[2] -= f * dz;
        }
      }
    }
    phi_s[k] = ph;
    grad_s[3 * k] = g[0];
    grad_s[3 * k + 1] = g[1];
    grad_s[3 * k + 2] = g[2];
  }
}

}  // namespace

// ------------------------------------------------------------------ C API
// Arrays of complex coefficients cross the boundary as interleaved (re, im)
// doubles, p*p entries per expansion, index n*(n+1)+m.
extern "C" {

int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

// xyzq: N x 4 doubles (x, y, z, q) in input order.
// mac: bit 0 circumscribed radius, bit 1 particle-fitted (tight) radius about
// the cube centre, bit 2 particle-fitted centres and radii (fitted).
int orc_build(const double* xyzq, int64_t N, int p, double theta, int ncrit, int mac_mode,
              void** out) {
  if (!xyzq || !out || N < 1 || p < 1 || p > 30 || !(theta > 0.0) || ncrit < 1) return -1;
  if (N > 2147483647ll) return -1;
  for (int64_t i = 0; i < 4 * N; ++i)
    if (!std::isfinite(xyzq[i])) return -2;
  Tree* t = new Tree();
  t->N = N;
  t->p = p;
  t->theta = theta;
  t->ncrit = ncrit;
  t->circumscribed = (mac_mode & 1) ? 1 : 0;
  t->tight = (mac_mode & 2) ? 1 : 0;
  t->fitted = (mac_mode & 4) ? 1 : 0;
  t->xyz.resize(3 * N);
  t->q.resize(N);
  for (int64_t i = 0; i < N; ++i) {
    t->xyz[3 * i] = xyzq[4 * i];
    t->xyz[3 * i + 1] = xyzq[4 * i + 1];
    t->xyz[3 * i + 2] = xyzq[4 * i + 2];
    t->q[i] = xyzq[4 * i + 3];
  }
  std::vector<uint64_t> key_in;
  root_and_keys(*t, key_in);
  // stable sort by key: ties keep input order
  t->perm.resize(N);
  std::iota(t->perm.begin(), t->perm.end(), 0);
  std::stable_sort(t->perm.begin(), t->perm.end(),
                   [&](int64_t a, int64_t b) { return key_in[a] < key_in[b]; });
  t->key_sorted.resize(N);
  for (int64_t i = 0; i < N; ++i) t->key_sorted[i] = key_in[t->perm[i]];
  build_cells(*t);
  if (t->fitted) fitted_centres(*t);
  else if (t->tight) tight_radii(*t);
  Traversal tr(*t);
  tr.visit(0, 0);
  const int ncell = (int)t->level.size();
  make_csr(ncell, tr.p2p, t->p2p_src, t->p2p_tgt, t->p2p_ptr);
  make_csr(ncell, tr.m2l, t->m2l_src, t->m2l_tgt, t->m2l_ptr);
  *out = t;
  return 0;
}

void orc_free(void* t) { delete (Tree*)t; }

// Expansion centre of every cell (ncell x 3 doubles).
int orc_centres(void* tp, double* out) {
  Tree& t = *(Tree*)tp;
  for (size_t c = 0; c < t.level.size(); ++c) cell_centre(t, (int)c, out + 3 * c);
  return 0;
}

// Expansion order of later evaluations.  The tree and the lists do not
// depend on it (Sec. III.A: P only sets the number of terms), so one build
// serves several orders.
int orc_set_order(void* tp, int p) {
  if (!tp || p < 1 || p > 30) return -1;
  Tree& t = *(Tree*)tp;
  t.p = p;
  t.M.clear();
  t.L.clear();
  return 0;
}

// info: ncell, nleaf, nlevel, n_p2p, n_m2l, p2p body pairs (excl. self)
int orc_info(void* tp, int64_t* info) {
  Tree& t = *(Tree*)tp;
  int64_t nleaf = 0, pairs = 0;
  for (size_t c = 0; c < t.level.size(); ++c) nleaf += t.nch[c] == 0;
  for (size_t e = 0; e < t.p2p_src.size(); ++e)
    pairs += (int64_t)(t.bend[t.p2p_src[e]] - t.bbeg[t.p2p_src[e]]) *
             (t.bend[t.p2p_tgt[e]] - t.bbeg[t.p2p_tgt[e]]);
  info[0] = (int64_t)t.level.size();
  info[1] = nleaf;
  info[2] = (int64_t)t.level_begin.size() - 1;
  info[3] = (int64_t)t.p2p_src.size();
  info[4] = (int64_t)t.m2l_src.size();
  info[5] = pairs - t.N;
  return 0;
}

// root: lo[3], hi[3], centre[3], H, corner r0[3]  (13 doubles)
int orc_root(void* tp, double* out) {
  Tree& t = *(Tree*)tp;
  for (int a = 0; a < 3; ++a) {
    out[a] = t.lo[a];
    out[3 + a] = t.hi[a];
    out[6 + a] = t.ctr[a];
    out[10 + a] = t.r0[a];
  }
  out[9] = t.H;
  return 0;
}

int orc_keys(void* tp, uint64_t* key_sorted, int64_t* perm) {
  Tree& t = *(Tree*)tp;
  std::memcpy(key_sorted, t.key_sorted.data(), sizeof(uint64_t) * t.N);
  std::memcpy(perm, t.perm.data(), sizeof(int64_t) * t.N);
  return 0;
}

// cells: 9 rows of ncell int32: level, ix, iy, iz, body_begin, body_end,
// child_begin (-1 for leaves), child_count, parent (-1 for the root)
int orc_cells(void* tp, int32_t* out) {
  Tree& t = *(Tree*)tp;
  const size_t n = t.level.size();
  const std::vector<int>* rows[9] = {&t.level, &t.ix, &t.iy, &t.iz, &t.bbeg,
                                     &t.bend, &t.cbeg, &t.nch, &t.parent};
  for (int r = 0; r < 9; ++r) std::memcpy(out + r * n, rows[r]->data(), sizeof(int32_t) * n);
  return 0;
}

int orc_lists(void* tp, int32_t* p2p_tgt, int32_t* p2p_src, int32_t* m2l_tgt, int32_t* m2l_src) {
  Tree& t = *(Tree*)tp;
  std::memcpy(p2p_tgt, t.p2p_tgt.data(), sizeof(int32_t) * t.p2p_tgt.size());
  std::memcpy(p2p_src, t.p2p_src.data(), sizeof(int32_t) * t.p2p_src.size());
  std::memcpy(m2l_tgt, t.m2l_tgt.data(), sizeof(int32_t) * t.m2l_tgt.size());
  std::memcpy(m2l_src, t.m2l_src.data(), sizeof(int32_t) * t.m2l_src.size());
  return 0;
}

// Evaluate potential and gradient.  xyz: N x 3 input-order positions for a
// frozen-tree evaluation, or null for the build's positions; q: N charges in
// input order, or null for the build's.  targets: input indices (null = all,
// outputs in input order).  mode: 1 near, 2 far, 3 both.
int orc_evaluate(void* tp, const double* xyz, const double* q, int mode, int64_t ntarget,
                 const int64_t* targets, double* phi, double* grad) {
  Tree& t = *(Tree*)tp;
  if (mode < 1 || mode > 3 || !phi || !grad) return -1;
  const int64_t N = t.N;
  std::vector<int64_t> inv(N);
  for (int64_t i = 0; i < N; ++i) inv[t.perm[i]] = i;
  std::vector<int64_t> tsorted;
  int64_t nt = N;
  if (targets) {
    nt = ntarget;
    tsorted.resize(nt);
    for (int64_t k = 0; k < nt; ++k) {
      if (targets[k] < 0 || targets[k] >= N) return -1;
      tsorted[k] = inv[targets[k]];
    }
  } else {
    tsorted.resize(N);
    for (int64_t k = 0; k < N; ++k) tsorted[k] = inv[k];  // output k = input body k
  }
  std::vector<double> ph(nt), gr(3 * nt);
  evaluate(t, xyz ? xyz : t.xyz.data(), q ? q : t.q.data(), mode, nt, tsorted.data(), ph.data(),
           gr.data());
  std::memcpy(phi, ph.data(), sizeof(double) * nt);
  std::memcpy(grad, gr.data(), sizeof(double) * 3 * nt);
  return 0;
}

// Expansions of the last evaluation: M and L, ncell x p*p complex each.
int orc_expansions(void* tp, double* M, double* L) {
  Tree& t = *(Tree*)tp;
  if (M) std::memcpy(M, t.M.data(), sizeof(cplx) * t.M.size());
  if (L) std::memcpy(L, t.L.data(), sizeof(cplx) * t.L.size());
  return 0;
}

// Adjoint of the scalar loss sum_i w_i phi_i with the tree frozen:
// dq = phi evaluated with charges w; dx = w grad phi_q + q grad phi_w.
int orc_backward(void* tp, const double* q, const double* w, double* dq, double* dx) {
  Tree& t = *(Tree*)tp;
  const int64_t N = t.N;
  const double* qq = q ? q : t.q.data();
  std::vector<double> pq(N), gq(3 * N), pw(N), gw(3 * N);
  int rc = orc_evaluate(tp, nullptr, qq, 3, 0, nullptr, pq.data(), gq.data());
  if (rc) return rc;
  rc = orc_evaluate(tp, nullptr, w, 3, 0, nullptr, pw.data(), gw.data());
  if (rc) return rc;
  for (int64_t i = 0; i < N; ++i) {
    dq[i] = pw[i];
    for (int a = 0; a < 3; ++a) dx[3 * i + a] = w[i] * gq[3 * i + a] + qq[i] * gw[3 * i + a];
  }
  return 0;
}

// Direct O(N^2) sum over all j != i (coincident bodies skipped) for the
// given target input indices (null = all).
int orc_direct(const double* xyzq, int64_t N, int64_t ntarget, const int64_t* targets,
               double* phi, double* grad) {
  const int64_t nt = targets ? ntarget : N;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t k = 0; k < nt; ++k) {
    const int64_t i = targets ? targets[k] : k;
    const double* xi = &xyzq[4 * i];
    double ph = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
    for (int64_t j = 0; j < N; ++j) {
      double dx = xi[0] - xyzq[4 * j], dy = xi[1] - xyzq[4 * j + 1], dz = xi[2] - xyzq[4 * j + 2];
      double r2 = dx * dx + dy * dy + dz * dz;
      if (r2 == 0.0) continue;
      double inv = 1.0 / std::sqrt(r2);
      double qi = xyzq[4 * j + 3] * inv;
      ph += qi;
      double f = qi * inv * inv;
      g0 -= f * dx;
      g1 -= f * dy;
      g2 -= f * dz;
    }
    phi[k] = ph;
    grad[3 * k] = g0;
    grad[3 * k + 1] = g1;
    grad[3 * k + 2] = g2;
  }
  return 0;
}

// ---- single operators (for the pins)
int orc_op_p2m(int p, const double* c, int nb, const double* xyzq, double* M) {
  std::vector<double> xyz(3 * nb), q(nb);
  for (int j = 0; j < nb; ++j) {
    xyz[3 * j] = xyzq[4 * j];
    xyz[3 * j + 1] = xyzq[4 * j + 1];
    xyz[3 * j + 2] = xyzq[4 * j + 2];
    q[j] = xyzq[4 * j + 3];
  }
  op_p2m(p, c, nb, xyz.data(), q.data(), (cplx*)M);
  return 0;
}
int orc_op_m2m(int p, const double* Mc, const double* cc, const double* cp, double* Mp) {
  op_m2m(p, (const cplx*)Mc, cc, cp, (cplx*)Mp);
  return 0;
}
int orc_op_m2l(int p, const double* M, const double* cA, const double* cB, double* L) {
  op_m2l(p, (const cplx*)M, cA, cB, (cplx*)L);
  return 0;
}
int orc_op_l2l(int p, const double* Lp, const double* cp, const double* cc, double* Lc) {
  op_l2l(p, (const cplx*)Lp, cp, cc, (cplx*)Lc);
  return 0;
}
// out: phi, gx, gy, gz (accumulated into)
int orc_op_l2p(int p, const double* L, const double* c, const double* x, double* out) {
  op_l2p(p, (const cplx*)L, c, x, &out[0], &out[1]);
  return 0;
}
int orc_op_m2p(int p, const double* M, const double* c, const double* x, double* out) {
  op_m2p(p, (const cplx*)M, c, x, &out[0], &out[1]);
  return 0;
}
// harmonics for the pins: U, T of p*p complex
int orc_harmonics(int p, const double* v, double* U, double* T) {
  if (U) regular(v, p, (cplx*)U);
  if (T) irregular(v, p, (cplx*)T);
  return 0;
}

}  // extern "C"
