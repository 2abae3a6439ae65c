// direct.cu -- double-precision direct summation at sampled targets, the
// reference the FMM's accuracy is reported against (the O(N^2) sum the FMM
// approximates; no tree involved).
#include "kernels.cuh"

namespace gbfmm {
namespace {

constexpr int kThreads = 256;

// One block per target: threads stride over the sources, block reduction in
// a fixed order.
__global__ void k_direct(const float4* __restrict__ xyzq, int64_t n, const int32_t* __restrict__ tg,
                         int64_t nt, double* __restrict__ pot, double* __restrict__ force) {
  const int64_t k = blockIdx.x;
  if (k >= nt) return;
  const int32_t i = tg[k];
  if (i < 0 || i >= n) {  // the whole block leaves: the target is not a body
    if (threadIdx.x == 0) {
      const double qnan = __longlong_as_double(0x7ff8000000000000ll);
      pot[k] = qnan;
      if (force) force[3 * k] = force[3 * k + 1] = force[3 * k + 2] = qnan;
    }
    return;
  }
  const float4 ti = xyzq[i];
  const double xi = ti.x, yi = ti.y, zi = ti.z;
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  for (int64_t j = threadIdx.x; j < n; j += kThreads) {
    const float4 b = xyzq[j];
    const double dx = (double)b.x - xi, dy = (double)b.y - yi, dz = (double)b.z - zi;
    const double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 == 0.0) continue;
    const double inv = 1.0 / sqrt(r2);
    const double qi = (double)b.w * inv;
    s0 += qi;
    const double f = qi * inv * inv;
    s1 += f * dx;
    s2 += f * dy;
    s3 += f * dz;
  }
  __shared__ double red[4][kThreads];
  red[0][threadIdx.x] = s0;
  red[1][threadIdx.x] = s1;
  red[2][threadIdx.x] = s2;
  red[3][threadIdx.x] = s3;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < 4; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pot[k] = red[0][0];
    if (force) {
      // grad phi = sum q (x_j - x_i) / r^3; force = -grad phi
      force[3 * k] = -red[1][0];
      force[3 * k + 1] = -red[2][0];
      force[3 * k + 2] = -red[3][0];
    }
  }
}

}  // namespace
}  // namespace gbfmm

extern "C" int fmm_direct_f64(const float* xyzq, int64_t n, const int32_t* targets, int64_t nt, double* pot,
                              double* force, fmm_stream stream) {
  if (!xyzq || !targets || !pot || n < 1 || nt < 0 || nt > 0x7fffffffll) return FMM_ERR_ARG;
  if (nt == 0) return FMM_OK;
  if (((uintptr_t)xyzq & 15) != 0) return FMM_ERR_ARG;
  try {
    gbfmm::k_direct<<<(unsigned)nt, gbfmm::kThreads, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const float4*>(xyzq), n, targets, nt, pot, force);
    GB_LAUNCH("k_direct");
  } catch (const gbfmm::Error& e) {
    return e.code;
  }
  return FMM_OK;
}
