// kernels.cuh -- launchers of the evaluation kernels (templated on the real
// type: float for the single-precision path, double for the double path).
#pragma once

#include <type_traits>

#include "common.cuh"

namespace gbfmm {

// Self-checking build (GBFMM_CHECKED): every data-dependent global access of
// the evaluation kernels is checked against the tree's array sizes (Lim); a
// violation is recorded in lim.rec (site, index, bound, count) and the access
// is skipped.
__device__ __forceinline__ bool in_range(long long i, long long n, int site, unsigned long long* rec) {
  if (i >= 0 && i < n) return true;
  if (rec) {
    if (atomicCAS(rec, 0ull, (unsigned long long)site) == 0ull) {
      rec[1] = (unsigned long long)i;
      rec[2] = (unsigned long long)n;
    }
    atomicAdd(rec + 3, 1ull);
  }
  return false;
}

#ifdef GBFMM_CHECKED
#define GB_LD(arr, i, n, site)                                                                     \
  (::gbfmm::in_range((long long)(i), (long long)(n), (site), lim.rec)                               \
       ? (arr)[(i)]                                                                                 \
       : typename std::remove_cv<typename std::remove_reference<decltype((arr)[0])>::type>::type())
#define GB_ST(arr, i, n, site, v)                                                   \
  do {                                                                              \
    if (::gbfmm::in_range((long long)(i), (long long)(n), (site), lim.rec)) (arr)[(i)] = (v); \
  } while (0)
#else
#define GB_LD(arr, i, n, site) ((arr)[(i)])
#define GB_ST(arr, i, n, site, v) ((arr)[(i)] = (v))
#endif

template <class R>
struct Vec4;
template <>
struct Vec4<float> {
  using type = float4;
};
template <>
struct Vec4<double> {
  using type = double4_32a;
};

template <class R> void launch_set_charges(fmm_tree* t, const R* q, cudaStream_t s);
template <class R> void launch_p2m(fmm_tree* t, cudaStream_t s);
template <class R> void launch_m2m(fmm_tree* t, int level, cudaStream_t s);
template <class R> void launch_l2l(fmm_tree* t, int level, cudaStream_t s);
template <class R> void launch_m2l_cuda_core(fmm_tree* t, cudaStream_t s);
template <class R> void launch_p2p(fmm_tree* t, cudaStream_t s);
// near-field work items of the single-precision kernel (after the lists)
void build_p2p_items(fmm_tree* t);
// mode 0: forward (pot, force out; gradient saved); mode 1: backward
// (a = dq, b = dx; the pass charges are the weights w).
template <class R> void launch_l2p_finalize(fmm_tree* t, int mode, R* a, R* b, cudaStream_t s);
void launch_m2l_tcgen05(fmm_tree* t, cudaStream_t s);
// FMM_FLAG_FITTED_CENTRES (fitted.cu): build-time centres and M2L CSR, and
// the per-child / per-pair translations
void build_fitted(fmm_tree* t);
template <class R> void launch_m2m_fit(fmm_tree* t, int level, cudaStream_t s);
template <class R> void launch_l2l_fit(fmm_tree* t, int level, cudaStream_t s);
template <class R> void launch_m2l_fit(fmm_tree* t, cudaStream_t s);
void launch_split_tf32(fmm_tree* t, cudaStream_t s);
void build_m2l_chunks(fmm_tree* t, int per);
// after the build's last read-back (chunk count in t->d_tail[3]): the count
// and the partial buffer
void finish_m2l_chunks(fmm_tree* t, int64_t nchunk);

}  // namespace gbfmm
