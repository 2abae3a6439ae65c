// m2l_cc.cu -- M2L on CUDA cores (Sec. II.A: the multipole of every
// well-separated cell is converted into the local expansion of the target;
// M2L and P2P take most of the run time, Sec. II.A).
//
// Work is organised by target tile (kTile targets) and translation operator:
// for one tile and one operator T_c the tile rows hold, per target, the one
// source that sits at that relative position (or nothing), so
//     L~[tile rows] += M~[sources] T_c^T
// is a small dense product.  One block per (tile, output chunk); thread r
// owns tile row r and OC output coefficients.  The contributions of the
// operators are summed in the working precision per operator and combined
// across operators with compensated (Kahan) addition.
#include "kernels.cuh"

namespace gbfmm {
namespace {

constexpr int KC = 32;  // input coefficients staged per step

template <class R, int OC>
__global__ void __launch_bounds__(kTile) k_m2l_cc(const int32_t* __restrict__ tile_tgt,
                                                  const int32_t* __restrict__ tile_eptr,
                                                  const int32_t* __restrict__ entry_class,
                                                  const int32_t* __restrict__ entry_src,
                                                  const R* __restrict__ ops, const R* __restrict__ M,
                                                  int K, int Kp, R* __restrict__ L, Lim lim) {
  __shared__ R Ms[kTile][KC + 1];
  __shared__ __align__(16) R OsT[KC][OC];
  const int tile = blockIdx.x;
  const int oc0 = blockIdx.y * OC;
  const int r = threadIdx.x;
  R acc[OC], comp[OC], part[OC];
#pragma unroll
  for (int o = 0; o < OC; ++o) acc[o] = comp[o] = (R)0;
  const int e0 = GB_LD(tile_eptr, tile, lim.ntile + 1, 201), e1 = GB_LD(tile_eptr, tile + 1, lim.ntile + 1, 202);
  for (int e = e0; e < e1; ++e) {
    const int cls = GB_LD(entry_class, e, lim.nentry, 203);
    int src = GB_LD(entry_src, (int64_t)e * kTile + r, lim.nentry * kTile, 204);
#ifdef GBFMM_CHECKED
    if (!in_range(cls, lim.nclass, 205, lim.rec)) continue;  // uniform over the block
    if (src >= 0 && !in_range(src, lim.ncell, 206, lim.rec)) src = -1;
#endif
    const R* op = ops + (int64_t)cls * Kp * Kp;
#pragma unroll
    for (int o = 0; o < OC; ++o) part[o] = (R)0;
    for (int k0 = 0; k0 < Kp; k0 += KC) {
      __syncthreads();
      const int kc = min(KC, Kp - k0);
      if (src >= 0) {
        const R* mrow = M + (int64_t)src * Kp + k0;
        for (int k = 0; k < kc; ++k) Ms[r][k] = mrow[k];
      } else {
        for (int k = 0; k < kc; ++k) Ms[r][k] = (R)0;
      }
      for (int i = r; i < OC * KC; i += kTile) {
        const int o = i / KC, k = i % KC;
        OsT[k][o] = (k < kc && oc0 + o < Kp) ? op[(int64_t)(oc0 + o) * Kp + k0 + k] : (R)0;
      }
      __syncthreads();
      for (int k = 0; k < kc; ++k) {
        const R m = Ms[r][k];
#pragma unroll
        for (int o = 0; o < OC; ++o) part[o] += m * OsT[k][o];
      }
    }
#pragma unroll
    for (int o = 0; o < OC; ++o) {
      const R y = part[o] - comp[o];
      const R tt = acc[o] + y;
      comp[o] = (tt - acc[o]) - y;
      acc[o] = tt;
    }
  }
  const int tgt = GB_LD(tile_tgt, (int64_t)tile * kTile + r, lim.ntile * kTile, 207);
  if (tgt < 0) return;
#ifdef GBFMM_CHECKED
  if (!in_range(tgt, lim.ncell, 208, lim.rec)) return;
#endif
  R* lrow = L + (int64_t)tgt * Kp + oc0;
#pragma unroll
  for (int o = 0; o < OC; ++o)
    if (oc0 + o < K) lrow[o] = acc[o];
}

}  // namespace

template <class R>
void launch_m2l_cuda_core(fmm_tree* t, cudaStream_t s) {
  if (t->ntile == 0) return;
  constexpr int OC = sizeof(R) == 4 ? 32 : 16;
  dim3 grid(t->ntile, (t->K + OC - 1) / OC);
  k_m2l_cc<R, OC><<<grid, kTile, 0, s>>>(t->tile_tgt, t->tile_eptr, t->entry_class, t->entry_src,
                                         (const R*)t->m2l_ops, (const R*)t->M, t->K, t->Kp, (R*)t->L, t->lim);
  GB_LAUNCH("k_m2l_cc");
}

template void launch_m2l_cuda_core<float>(fmm_tree*, cudaStream_t);
template void launch_m2l_cuda_core<double>(fmm_tree*, cudaStream_t);

}  // namespace gbfmm
