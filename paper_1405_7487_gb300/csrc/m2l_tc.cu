// m2l_tc.cu -- M2L on the 5th-generation tensor cores (tcgen05), single
// precision through three TF32 products.
//
// M2L converts the multipole of each well-separated source into the local
// expansion of the target (Sec. II.A; with P2P it takes most of the run
// time).  Targets are tiled 128 at a time; for one tile and one translation
// operator T_c (an entry of the plan) the 128 rows hold the source of each
// target at that relative position, so the entry is the product
//     L~[128 x Kp] += M~_src[128 x Kp] . T_c^T[Kp x Kp]
// (M = 128 rows, N = Kp outputs, K = Kp inputs).
//
// Precision: every operand x is split into hi = tf32(x) and lo = tf32(x - hi)
// (both rounded to nearest, so the tensor core sees them exactly) and each
// entry issues hi*hi + lo*hi + hi*lo.  The entries of a tile are cut into
// chunks of a few entries; each chunk accumulates in TMEM (fp32) and is
// written out as a partial, and the partials of a tile are added with
// compensated (Kahan) summation in a fixed order (k_m2l_reduce).  Short
// chunks bound the rounding of the fp32 tensor-core accumulation.
//
// Pipeline (one CTA per chunk, 160 threads), stages of one 32-element
// k-block in the 128-byte-swizzled K-major layout the MMA descriptors
// describe:
//   warps 0-3  producers: cp.async 16-byte copies of the 128 gathered source
//              rows (hi and lo); each thread publishes its part of a stage
//              with cp.async.mbarrier.arrive (the arrival on the stage's
//              "full" barrier fires when its copies land).  Thread 0 also
//              loads the operator's k-block (Kp rows, hi and lo) with two
//              tiled TMA copies that complete on the stage's operator
//              barrier.  Up to nstage stages are in flight.  Then the
//              epilogue (TMEM -> the chunk's partial).
//   warp 4     TMEM allocation; one elected lane waits for both barriers of
//              a stage, fences the generic-proxy writes against the tensor
//              core's async-proxy reads, issues the stage's MMAs and commits
//              them to the stage's "empty" barrier.
// Every wait is bounded; a wait that gives up sets the error flag, the
// roles drain and the TMEM is released.
#include <algorithm>
#include <cstdlib>
#include <vector>

#include "kernels.cuh"
#include "mbarrier.cuh"

namespace gbfmm {

// Trace build (-DGBFMM_M2L_TRACE, libgbfmm_traced.so): the quad engine adds
// the clock64 cycles its roles spend waiting and working to g_m2l_trace
// (fmm_debug_m2l_trace reads and clears them).  Slots:
//   0 producers: wait for a free source stage (thread 0)
//   1 producers: wait for a free operator stage (thread 0)
//   2 MMA thread: block start to its first wait
//   3 MMA thread: its last commit to the end of the block
//   5 MMA: wait for an operator stage     6 MMA: wait for a source stage
//   7 MMA: issue + commit                11 whole block     12 blocks
//  13 producers: wait for the last MMA   14 epilogue
// (sums over all blocks).
#ifdef GBFMM_M2L_TRACE
__device__ unsigned long long g_m2l_trace[16];
#define M2L_T0(v) const long long v = clock64()
#define M2L_ADD(slot, t0, cond) \
  if (cond) atomicAdd(&g_m2l_trace[slot], (unsigned long long)(clock64() - (t0)))
#else
#define M2L_T0(v)
#define M2L_ADD(slot, t0, cond)
#endif

namespace {

constexpr int kProducers = 128;
constexpr int kThreadsTC = 160;
constexpr int kMaxStages = 8;

constexpr int kKB = 32;               // fp32 elements per k-block (128 bytes per row)
constexpr int kRowB = kKB * 4;        // bytes per row of a k-block
constexpr int kStageA = 128 * kRowB;  // bytes of one 128-row operand block

// Byte offset of 16-byte chunk c (0..7) of row r in a [rows][128 B] block
// with the 128-byte swizzle: address bits [4,6] are XORed with bits [7,9],
// i.e. the chunk index with r % 8 (8-row groups of 1024 bytes).  TMA writes
// the same pattern for a 128-byte-wide box with CU_TENSOR_MAP_SWIZZLE_128B.
__device__ __forceinline__ uint32_t swz(int r, int c) {
  return (uint32_t)((r << 7) + (((c ^ r) & 7) << 4));
}

// UMMA shared-memory descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), sm_100 descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;              // LBO (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;    // SBO
  d |= (uint64_t)1 << 46;              // version
  d |= (uint64_t)2 << 61;              // SWIZZLE_128B
  return d;
}

// 2-D tiled TMA load of the box at (x, y) into dst; completes on bar.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// The same with an L2 cache policy (createpolicy) for the loaded lines.
__device__ __forceinline__ void tma_load_2d_hint(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar,
                                                 uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, "
      "{%2, %3}], [%4], %5;\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar), "l"(policy)
      : "memory");
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Instruction descriptor, kind::tf32: D fp32, A and B tf32, both K-major,
// N = n, M = 128.
__device__ __forceinline__ uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
               : "memory");
}

__global__ void __launch_bounds__(kThreadsTC, 1)
    k_m2l_tc(const __grid_constant__ CUtensorMap tm_ops_hi, const __grid_constant__ CUtensorMap tm_ops_lo,
             const int4* __restrict__ chunks, const int32_t* __restrict__ entry_class,
             const int32_t* __restrict__ entry_src, const float* __restrict__ Mhi, const float* __restrict__ Mlo,
             int Kp, int nstage, int tmem_cols, float* __restrict__ part, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t bar_full[kMaxStages], bar_opfull[kMaxStages], bar_empty[kMaxStages], bar_done;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;

  // 1024-byte aligned stage buffers
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const int stageB = Kp * kRowB;
  const int stage_bytes = 2 * kStageA + 2 * stageB;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // chunk = (tile, first entry, end entry, partial slot): a bounded run of
  // the tile's entries, accumulated in TMEM and written as one partial sum
  const int4 ch = chunks[blockIdx.x];
  const int e0 = ch.y, e1 = ch.z;
  const int nkb = (Kp + kKB - 1) / kKB;
  const int nit = (e1 - e0) * nkb;

  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < nstage; ++s) {
      mbar_init(smem_u32(&bar_full[s]), kProducers);  // the producers' cp.async arrivals
      mbar_init(smem_u32(&bar_opfull[s]), 1);         // the operator TMA (expect-tx)
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    mbar_init(smem_u32(&bar_done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (warp < 4) {
    // ---------------------------------------------------------- producers
    // A (the gathered source rows): thread r moves 16-byte chunk (r % 8) of
    // rows r / 8 + 16 i, so eight neighbouring threads read one 128-byte row
    // segment and write one swizzled line; each thread's part of a stage is
    // published by cp.async.mbarrier.arrive, which fires when its copies
    // have landed.  B (the operator's k-block, Kp rows x 128 bytes, hi and
    // lo): two tiled TMA loads issued by thread 0, completing on the stage's
    // operator barrier through expect-tx.  The producers run ahead by up to
    // nstage stages; the next entry's source rows are loaded while the
    // current entry is copied.
    const int r = tid;
    const int c8 = r & 7, r8 = r >> 3;
    const uint32_t b_bytes = 2u * (uint32_t)stageB;
    int src[8], nsrc[8];
    int cls = 0, ncls = 0;
    int tma_issued = 0;  // thread 0: operator loads issued
    auto fetch = [&](int e, int (&to)[8], int& tc) {
#pragma unroll
      for (int i = 0; i < 8; ++i) to[i] = __ldg(entry_src + (int64_t)e * kTile + r8 + 16 * i);
      tc = __ldg(entry_class + e);
    };
    if (nit > 0) fetch(e0, nsrc, ncls);
    for (int it = 0; it < nit; ++it) {
      const int e = e0 + it / nkb, kb = it % nkb;
      const int s = it % nstage, round = it / nstage;
      if (kb == 0) {
#pragma unroll
        for (int i = 0; i < 8; ++i) src[i] = nsrc[i];
        cls = ncls;
        if (e + 1 < e1) fetch(e + 1, nsrc, ncls);
      }
      if (round > 0 && !mbar_wait(smem_u32(&bar_empty[s]), (round - 1) & 1, &abort_flag)) break;
      const uint32_t sb = base + s * stage_bytes;
      const int k0 = kb * kKB;
      if (r == 0) {
        // the box is 32 columns wide; columns past Kp (last k-block) read as
        // zeros and are not used by the MMAs
        const uint32_t ob = smem_u32(&bar_opfull[s]);
        mbar_arrive_expect_tx(ob, b_bytes);
        tma_load_2d(sb + 2 * kStageA, &tm_ops_hi, k0, cls * Kp, ob);
        tma_load_2d(sb + 2 * kStageA + stageB, &tm_ops_lo, k0, cls * Kp, ob);
        tma_issued = it + 1;
      }
      const int nch = min(kKB, Kp - k0) / 4;  // 16-byte chunks in this k-block
      if (c8 < nch) {
        // A rows: the source multipole of each tile row (zeros for an empty row)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int row = r8 + 16 * i;
          const int64_t off = (int64_t)(src[i] >= 0 ? src[i] : 0) * Kp + k0 + 4 * c8;
          const int bytes = src[i] >= 0 ? 16 : 0;
          cp_async16(sb + swz(row, c8), Mhi + off, bytes);
          cp_async16(sb + kStageA + swz(row, c8), Mlo + off, bytes);
        }
      }
      asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(smem_u32(&bar_full[s]))
                   : "memory");
    }
    // no copy may still be in flight when the CTA ends: the thread's own
    // cp.async copies, and (thread 0, after an abort) the last operator load
    cp_async_wait<0>();
    if (r == 0)  // every operator load that may still be in flight
      for (int i = max(0, tma_issued - nstage); i < tma_issued; ++i)
        if (!mbar_drain(smem_u32(&bar_opfull[i % nstage]), (i / nstage) & 1)) atomicOr(err, kErrDrain);
    // ------------------------------------------------------------ epilogue
    const bool ok = nit > 0 && mbar_wait(smem_u32(&bar_done), 0, &abort_flag);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (ok || nit == 0) {
      // partial slot ch.w, column-major ([Kp][128]): a warp's store of one
      // column is 128 contiguous bytes
      float* pcol = part + (int64_t)ch.w * kTile * Kp + r;
      for (int c0 = 0; c0 < Kp; c0 += 16) {
        uint32_t v[16];
        if (nit > 0) {
          const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
              "[%16];\n"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
              : "r"(taddr)
              : "memory");
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        } else {
          for (int k = 0; k < 16; ++k) v[k] = 0u;
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) __stcs(pcol + (int64_t)(c0 + k) * kTile, __uint_as_float(v[k]));
      }
    }
  } else if (lane == 0) {
    // ---------------------------------------------------------------- MMA
    const uint32_t idesc = idesc_tf32(Kp);
    bool ok = true;
    for (int it = 0; it < nit; ++it) {
      const int kb = it % nkb;
      const int s = it % nstage, round = it / nstage;
      if (!mbar_wait(smem_u32(&bar_full[s]), round & 1, &abort_flag) ||
          !mbar_wait(smem_u32(&bar_opfull[s]), round & 1, &abort_flag)) {
        ok = false;
        break;
      }
      // A was written through the generic proxy (cp.async); make it visible
      // to the tensor core's async-proxy reads
      fence_async_smem();
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t sb = base + s * stage_bytes;
      const int nks = min(kKB, Kp - kb * kKB) / 8;  // tf32 k-steps of 8 elements
      for (int ks = 0; ks < nks; ++ks) {
        const uint32_t off = ks * 32;
        const uint64_t ah = smem_desc(sb + off), al = smem_desc(sb + kStageA + off);
        const uint64_t bh = smem_desc(sb + 2 * kStageA + off), bl = smem_desc(sb + 2 * kStageA + stageB + off);
        const uint32_t first = (it == 0 && ks == 0) ? 0u : 1u;
        mma_tf32(tmem, ah, bh, idesc, first);
        mma_tf32(tmem, al, bh, idesc, 1u);
        mma_tf32(tmem, ah, bl, idesc, 1u);
      }
      mma_commit(smem_u32(&bar_empty[s]));
    }
    // tracks every MMA issued, also after an abort, so that the TMEM is
    // released only when they are done
    if (nit > 0) mma_commit(smem_u32(&bar_done));
    if (!ok) abort_flag = 1;
  }
  // drain: the last commits must land before the TMEM is released
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (abort_flag && tid == 0) atomicOr(err, kErrWait);
  if (warp == 4) {
    if (abort_flag && nit > 0) {
      // wait (bounded) for the MMAs that were issued before the TMEM is
      // released; if they are not seen to finish, the release still happens
      // (an unreleased allocation would block every later block on this SM)
      // and the error word says so
      if (!mbar_drain(smem_u32(&bar_done), 0) && lane == 0) atomicOr(err, kErrDrain);
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tmem_cols) : "memory");
  }
}

// Single-tile engine that folds after every entry (Kp <= 256, so that two
// accumulators of tmem_cols columns fit the 512 TMEM columns).  The MMAs of
// one entry accumulate in A (columns 0 ..), restarting at the entry's first
// k-step; when they are done (bar_acc), four fold warps add A into B
// (columns tmem_cols ..) with FP32 adds in registers and tell the MMA thread
// that A is free (bar_free), and the last fold's B is the chunk's partial.
// Each FP32 accumulation inside the tensor core then spans one entry's
// k-steps instead of the chunk's, which is what sets the single-precision
// error floor at high orders; the cost is that an entry's MMAs wait for the
// fold of the one before.  Warps 0-3 produce as in k_m2l_tc, warp 4 issues
// the MMAs, warps 5-8 fold and write the partial.
constexpr int kThreadsFold = 288;

__device__ __forceinline__ void mbar_arrive1(uint32_t bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n" ::"r"(
          taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}

__global__ void __launch_bounds__(kThreadsFold, 1)
    k_m2l_tc_fold(const __grid_constant__ CUtensorMap tm_ops_hi, const __grid_constant__ CUtensorMap tm_ops_lo,
                  const int4* __restrict__ chunks, const int32_t* __restrict__ entry_class,
                  const int32_t* __restrict__ entry_src, const float* __restrict__ Mhi, const float* __restrict__ Mlo,
                  int Kp, int nstage, int tmem_cols, float* __restrict__ part, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t bar_full[kMaxStages], bar_opfull[kMaxStages], bar_empty[kMaxStages], bar_done, bar_acc,
      bar_free;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;

  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const int stageB = Kp * kRowB;
  const int stage_bytes = 2 * kStageA + 2 * stageB;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int4 ch = chunks[blockIdx.x];
  const int e0 = ch.y, e1 = ch.z;
  const int nkb = (Kp + kKB - 1) / kKB;
  const int ne = e1 - e0;
  const int nit = ne * nkb;

  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < nstage; ++s) {
      mbar_init(smem_u32(&bar_full[s]), kProducers);
      mbar_init(smem_u32(&bar_opfull[s]), 1);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    mbar_init(smem_u32(&bar_done), 1);
    mbar_init(smem_u32(&bar_acc), 1);
    mbar_init(smem_u32(&bar_free), 4);  // one arrival per fold warp
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                 "r"(2 * tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (warp < 4) {
    // ---------------------------------------------------------- producers
    // (as in k_m2l_tc)
    const int r = tid;
    const int c8 = r & 7, r8 = r >> 3;
    const uint32_t b_bytes = 2u * (uint32_t)stageB;
    int src[8], nsrc[8];
    int cls = 0, ncls = 0;
    int tma_issued = 0;
    auto fetch = [&](int e, int (&to)[8], int& tc) {
#pragma unroll
      for (int i = 0; i < 8; ++i) to[i] = __ldg(entry_src + (int64_t)e * kTile + r8 + 16 * i);
      tc = __ldg(entry_class + e);
    };
    if (nit > 0) fetch(e0, nsrc, ncls);
    for (int it = 0; it < nit; ++it) {
      const int e = e0 + it / nkb, kb = it % nkb;
      const int s = it % nstage, round = it / nstage;
      if (kb == 0) {
#pragma unroll
        for (int i = 0; i < 8; ++i) src[i] = nsrc[i];
        cls = ncls;
        if (e + 1 < e1) fetch(e + 1, nsrc, ncls);
      }
      if (round > 0 && !mbar_wait(smem_u32(&bar_empty[s]), (round - 1) & 1, &abort_flag)) break;
      const uint32_t sb = base + s * stage_bytes;
      const int k0 = kb * kKB;
      if (r == 0) {
        const uint32_t ob = smem_u32(&bar_opfull[s]);
        mbar_arrive_expect_tx(ob, b_bytes);
        tma_load_2d(sb + 2 * kStageA, &tm_ops_hi, k0, cls * Kp, ob);
        tma_load_2d(sb + 2 * kStageA + stageB, &tm_ops_lo, k0, cls * Kp, ob);
        tma_issued = it + 1;
      }
      const int nch = min(kKB, Kp - k0) / 4;
      if (c8 < nch) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int row = r8 + 16 * i;
          const int64_t off = (int64_t)(src[i] >= 0 ? src[i] : 0) * Kp + k0 + 4 * c8;
          const int bytes = src[i] >= 0 ? 16 : 0;
          cp_async16(sb + swz(row, c8), Mhi + off, bytes);
          cp_async16(sb + kStageA + swz(row, c8), Mlo + off, bytes);
        }
      }
      asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(smem_u32(&bar_full[s]))
                   : "memory");
    }
    cp_async_wait<0>();
    if (r == 0)
      for (int i = max(0, tma_issued - nstage); i < tma_issued; ++i)
        if (!mbar_drain(smem_u32(&bar_opfull[i % nstage]), (i / nstage) & 1)) atomicOr(err, kErrDrain);
  } else if (warp == 4) {
    // ---------------------------------------------------------------- MMA
    if (lane == 0) {
      const uint32_t idesc = idesc_tf32(Kp);
      bool ok = true;
      for (int it = 0; it < nit && ok; ++it) {
        const int j = it / nkb, kb = it % nkb;
        const int s = it % nstage, round = it / nstage;
        if (kb == 0 && j > 0) {
          // A is free once the fold of entry j - 1 has read it
          if (!mbar_wait(smem_u32(&bar_free), (j - 1) & 1, &abort_flag)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        }
        if (!mbar_wait(smem_u32(&bar_full[s]), round & 1, &abort_flag) ||
            !mbar_wait(smem_u32(&bar_opfull[s]), round & 1, &abort_flag)) {
          ok = false;
          break;
        }
        fence_async_smem();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t sb = base + s * stage_bytes;
        const int nks = min(kKB, Kp - kb * kKB) / 8;
        for (int ks = 0; ks < nks; ++ks) {
          const uint32_t off = ks * 32;
          const uint64_t ah = smem_desc(sb + off), al = smem_desc(sb + kStageA + off);
          const uint64_t bh = smem_desc(sb + 2 * kStageA + off), bl = smem_desc(sb + 2 * kStageA + stageB + off);
          const uint32_t first = (kb == 0 && ks == 0) ? 0u : 1u;  // A restarts with each entry
          mma_tf32(tmem, ah, bh, idesc, first);
          mma_tf32(tmem, al, bh, idesc, 1u);
          mma_tf32(tmem, ah, bl, idesc, 1u);
        }
        mma_commit(smem_u32(&bar_empty[s]));
        if (kb == nkb - 1) mma_commit(smem_u32(&bar_acc));  // entry j's sum is in A
      }
      if (nit > 0) mma_commit(smem_u32(&bar_done));
      if (!ok) abort_flag = 1;
    }
  } else {
    // --------------------------------------------------- fold and partial
    // warp w reaches the TMEM lanes 32 (w % 4) ..; its thread owns tile row
    // 32 (w % 4) + lane
    const int q = warp & 3;
    const uint32_t lanes = (uint32_t)(q * 32) << 16;
    const uint32_t ta = tmem + lanes, tb = tmem + lanes + (uint32_t)tmem_cols;
    bool ok = true;
    for (int j = 0; j < ne; ++j) {
      if (!mbar_wait(smem_u32(&bar_acc), j & 1, &abort_flag)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      for (int c0 = 0; c0 < Kp; c0 += 16) {
        uint32_t a[16], b[16];
        tmem_ld16(ta + (uint32_t)c0, a);
        if (j > 0) tmem_ld16(tb + (uint32_t)c0, b);
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        if (j > 0)
#pragma unroll
          for (int k = 0; k < 16; ++k) a[k] = __float_as_uint(__uint_as_float(a[k]) + __uint_as_float(b[k]));
        tmem_st16(tb + (uint32_t)c0, a);
      }
      asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive1(smem_u32(&bar_free));
    }
    if (ok) {
      // partial slot ch.w, column-major ([Kp][128])
      float* pcol = part + (int64_t)ch.w * kTile * Kp + q * 32 + lane;
      for (int c0 = 0; c0 < Kp; c0 += 16) {
        uint32_t v[16];
        if (ne > 0) {
          tmem_ld16(tb + (uint32_t)c0, v);
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        } else {
          for (int k = 0; k < 16; ++k) v[k] = 0u;
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) __stcs(pcol + (int64_t)(c0 + k) * kTile, __uint_as_float(v[k]));
      }
    }
  }
  // drain: the last commits must land before the TMEM is released
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (abort_flag && tid == 0) atomicOr(err, kErrWait);
  if (warp == 4) {
    if (abort_flag && nit > 0) {
      if (!mbar_drain(smem_u32(&bar_done), 0) && lane == 0) atomicOr(err, kErrDrain);
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(2 * tmem_cols)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// Quad engine (Kp <= 128): one CTA takes four tiles of the same octant
// together.  The tiles' class lists are merged into quad entries (class, the
// entry of each tile or -1); per quad entry and k-block the operator's
// k-block is loaded once (TMA, two stages) and multiplied with the source
// rows of every tile that has the class (cp.async, kAStages stages of
// 128 rows), each tile accumulating in its own quarter of the TMEM (128
// columns).  So the operator bytes per tile entry drop four-fold, and the
// source-row stages can run deeper than the combined stages of the
// single-tile engine.  Chunks of up to kM2LChunk quad entries per CTA; the
// partial of (chunk, tile) is written column-major, zeros for a tile without
// entries in the chunk.
constexpr int kQuad = 4;
constexpr int kMaxAStages = 6;
constexpr int kQuadMaxKp = 128;  // four 128-column TMEM accumulators

// The single-tile engine folds after every entry (k_m2l_tc_fold) unless
// GBFMM_M2L_FOLD=0 (a knob for measuring what the fold costs and gains).
bool m2l_fold_enabled() {
  static const bool on = [] {
    const char* env = getenv("GBFMM_M2L_FOLD");
    return !(env && atoi(env) == 0);
  }();
  return on;
}

// GBFMM_M2L_SINGLE=1 selects the single-tile engine at every Kp (tuning and
// cross-checking knob)
bool m2l_single_tile_forced() {
  static const bool on = [] {
    const char* env = getenv("GBFMM_M2L_SINGLE");
    return env && atoi(env) == 1;
  }();
  return on;
}

__global__ void __launch_bounds__(kThreadsTC, 1)
    k_m2l_tc4(const __grid_constant__ CUtensorMap tm_ops_hi, const __grid_constant__ CUtensorMap tm_ops_lo,
              const int4* __restrict__ chunks, const int32_t* __restrict__ quad_class,
              const int4* __restrict__ quad_entry, const int32_t* __restrict__ entry_src,
              const float* __restrict__ Mhi, const float* __restrict__ Mlo, int Kp, int Kin, int nastage,
              float* __restrict__ part, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t bar_bfull[2], bar_bempty[2], bar_afull[kMaxAStages], bar_aempty[kMaxAStages], bar_done;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;

  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const int stageB = Kp * kRowB;           // one of hi / lo
  const uint32_t bbase = base;             // 2 operator stages of 2 * stageB
  const uint32_t abase = base + 4 * stageB;  // nastage source stages of 2 * kStageA

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  M2L_T0(t_block);
  const int4 ch = chunks[blockIdx.x];
  const int j0 = ch.y, j1 = ch.z;
  // the inputs span Kin = K rounded up to the 8-element k-step (columns
  // K .. Kp of M and of the operators are zero); the outputs span Kp
  const int nkb = (Kin + kKB - 1) / kKB;

  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < 2; ++s) {
      mbar_init(smem_u32(&bar_bfull[s]), 1);
      mbar_init(smem_u32(&bar_bempty[s]), 1);
    }
    for (int s = 0; s < nastage; ++s) {
      mbar_init(smem_u32(&bar_afull[s]), kProducers);
      mbar_init(smem_u32(&bar_aempty[s]), 1);
    }
    mbar_init(smem_u32(&bar_done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (warp < 4) {
    // ---------------------------------------------------------- producers
    const int r = tid;
    const int c8 = r & 7, r8 = r >> 3;
    // the next quad entry's class, entries and source rows are loaded while
    // the current one is copied
    int src[kQuad][8], nsrc[kQuad][8];
    int ncls = 0, used = 0;
    int4 ne4 = make_int4(-1, -1, -1, -1);
    auto fetch = [&](int j) {
      ncls = __ldg(quad_class + j);
      ne4 = __ldg(quad_entry + j);
      const int ev[kQuad] = {ne4.x, ne4.y, ne4.z, ne4.w};
#pragma unroll
      for (int q = 0; q < kQuad; ++q)
        if (ev[q] >= 0) {
#pragma unroll
          for (int i = 0; i < 8; ++i) nsrc[q][i] = __ldg(entry_src + (int64_t)ev[q] * kTile + r8 + 16 * i);
        }
    };
    int bi = 0, ai = 0;
    int tma_issued = 0;  // thread 0: operator stages issued
    bool stop = false;
    // operator k-blocks stay in L2 (evict-last): every tile group that has
    // the class reads them again
    uint64_t policy = 0;
    if (r == 0) asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(policy));
    if (j1 > j0) fetch(j0);
    for (int j = j0; j < j1 && !stop; ++j) {
      const int cls = ncls;
      const int ev[kQuad] = {ne4.x, ne4.y, ne4.z, ne4.w};
#pragma unroll
      for (int q = 0; q < kQuad; ++q) {
        if (ev[q] < 0) continue;
        used |= 1 << q;
#pragma unroll
        for (int i = 0; i < 8; ++i) src[q][i] = nsrc[q][i];
      }
      if (j + 1 < j1) fetch(j + 1);
      for (int kb = 0; kb < nkb && !stop; ++kb, ++bi) {
        const int k0 = kb * kKB;
        if (r == 0) {
          const int bs = bi & 1, bround = bi >> 1;
          M2L_T0(t1);
          if (bround > 0 && !mbar_wait(smem_u32(&bar_bempty[bs]), (bround - 1) & 1, &abort_flag)) {
            stop = true;
            break;
          }
          M2L_ADD(1, t1, true);
          // the box is 32 columns wide; columns past Kp (last k-block) read
          // as zeros and are not used by the MMAs
          const uint32_t fb = smem_u32(&bar_bfull[bs]);
          const uint32_t sb = bbase + bs * 2 * stageB;
          mbar_arrive_expect_tx(fb, 2u * (uint32_t)stageB);
          tma_load_2d_hint(sb, &tm_ops_hi, k0, cls * Kp, fb, policy);
          tma_load_2d_hint(sb + stageB, &tm_ops_lo, k0, cls * Kp, fb, policy);
          tma_issued = bi + 1;
        }
        const int nch = min(kKB, Kin - k0) / 4;  // 16-byte chunks in this k-block
#pragma unroll
        for (int q = 0; q < kQuad; ++q) {
          if (ev[q] < 0) continue;
          const int as = ai % nastage, around = ai / nastage;
          M2L_T0(t0);
          if (around > 0 && !mbar_wait(smem_u32(&bar_aempty[as]), (around - 1) & 1, &abort_flag)) {
            stop = true;
            break;
          }
          M2L_ADD(0, t0, r == 0);
          const uint32_t sa = abase + as * 2 * kStageA;
          if (c8 < nch) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const int row = r8 + 16 * i;
              const int sidx = src[q][i];
              const int64_t off = (int64_t)(sidx >= 0 ? sidx : 0) * Kp + k0 + 4 * c8;
              const int bytes = sidx >= 0 ? 16 : 0;
              cp_async16(sa + swz(row, c8), Mhi + off, bytes);
              cp_async16(sa + kStageA + swz(row, c8), Mlo + off, bytes);
            }
          }
          asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(smem_u32(&bar_afull[as]))
                       : "memory");
          ++ai;
        }
      }
    }
    // no copy may still be in flight when the CTA ends
    cp_async_wait<0>();
    if (r == 0)  // both operator stages may still be in flight
      for (int i = max(0, tma_issued - 2); i < tma_issued; ++i)
        if (!mbar_drain(smem_u32(&bar_bfull[i & 1]), (i >> 1) & 1)) atomicOr(err, kErrDrain);
    // ------------------------------------------------------------ epilogue
    M2L_T0(t13);
    const bool ok = j1 > j0 && mbar_wait(smem_u32(&bar_done), 0, &abort_flag);
    M2L_ADD(13, t13, r == 0);
    M2L_T0(t14);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (ok) {
      for (int q = 0; q < kQuad; ++q) {
        // partial (chunk ch.w, tile q), column-major ([Kp][128])
        float* pcol = part + ((int64_t)ch.w * kQuad + q) * kTile * Kp + r;
        for (int c0 = 0; c0 < Kp; c0 += 16) {
          uint32_t v[16];
          if (used & (1 << q)) {
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(q * 128 + c0);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];\n"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(taddr)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
          } else {
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] = 0u;
          }
#pragma unroll
          for (int k = 0; k < 16; ++k) __stcs(pcol + (int64_t)(c0 + k) * kTile, __uint_as_float(v[k]));
        }
      }
    }
    M2L_ADD(14, t14, r == 0);
  } else if (lane == 0) {
    // ---------------------------------------------------------------- MMA
    M2L_ADD(2, t_block, true);
    const uint32_t idesc = idesc_tf32(Kp);
    bool ok = true;
    bool first[kQuad] = {true, true, true, true};
    int bi = 0, ai = 0;
    for (int j = j0; j < j1 && ok; ++j) {
      const int4 e4 = __ldg(quad_entry + j);
      const int ev[kQuad] = {e4.x, e4.y, e4.z, e4.w};
      for (int kb = 0; kb < nkb && ok; ++kb, ++bi) {
        const int bs = bi & 1, bround = bi >> 1;
        M2L_T0(t5);
        if (!mbar_wait(smem_u32(&bar_bfull[bs]), bround & 1, &abort_flag)) {
          ok = false;
          break;
        }
        M2L_ADD(5, t5, true);
        const uint32_t sb = bbase + bs * 2 * stageB;
        const int nks = min(kKB, Kin - kb * kKB) / 8;  // tf32 k-steps of 8 elements
#pragma unroll
        for (int q = 0; q < kQuad; ++q) {
          if (ev[q] < 0) continue;
          const int as = ai % nastage, around = ai / nastage;
          M2L_T0(t6);
          if (!mbar_wait(smem_u32(&bar_afull[as]), around & 1, &abort_flag)) {
            ok = false;
            break;
          }
          M2L_ADD(6, t6, true);
          M2L_T0(t7);
          // the source rows were written through the generic proxy (cp.async)
          fence_async_smem();
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const uint32_t sa = abase + as * 2 * kStageA;
          const uint32_t acc = tmem + (uint32_t)(q * 128);
          for (int ks = 0; ks < nks; ++ks) {
            const uint32_t off = ks * 32;
            const uint64_t ah = smem_desc(sa + off), al = smem_desc(sa + kStageA + off);
            const uint64_t bh = smem_desc(sb + off), bl = smem_desc(sb + stageB + off);
            mma_tf32(acc, ah, bh, idesc, first[q] ? 0u : 1u);
            first[q] = false;
            mma_tf32(acc, al, bh, idesc, 1u);
            mma_tf32(acc, ah, bl, idesc, 1u);
          }
          mma_commit(smem_u32(&bar_aempty[as]));
          ++ai;
          M2L_ADD(7, t7, true);
        }
        // the operator stage is free once the MMAs that read it are done
        mma_commit(smem_u32(&bar_bempty[bs]));
      }
    }
    // tracks every MMA issued, also after an abort
    if (j1 > j0) mma_commit(smem_u32(&bar_done));
    if (!ok) abort_flag = 1;
  }
  M2L_T0(t_tail);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  M2L_ADD(3, t_tail, warp == 4 && lane == 0);
  if (abort_flag && tid == 0) atomicOr(err, kErrWait);
  M2L_ADD(11, t_block, tid == 0);
#ifdef GBFMM_M2L_TRACE
  if (tid == 0) atomicAdd(&g_m2l_trace[12], 1ull);
#endif
  if (warp == 4) {
    if (abort_flag && j1 > j0) {
      if (!mbar_drain(smem_u32(&bar_done), 0) && lane == 0) atomicOr(err, kErrDrain);
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(512) : "memory");
  }
}

// L rows of one tile = compensated (Kahan) sum of the partials of its
// quad's chunks, in chunk order.  Thread per (coefficient, row); the
// partials are loaded eight chunks at a time so that the loads overlap.
__global__ void k_m2l_reduce4(const int32_t* __restrict__ tile_tgt, const int32_t* __restrict__ quad_cptr,
                              const float* __restrict__ part, int K, int Kp, float* __restrict__ L) {
  const int tile = blockIdx.x;
  const int q = tile / kQuad, lq = tile % kQuad;
  const int c0 = quad_cptr[q], c1 = quad_cptr[q + 1];
  const int64_t cstride = (int64_t)kQuad * Kp * kTile;  // floats between chunks
  // thread per (coefficient, four consecutive rows): 16-byte loads of the
  // column-major partials, four compensated sums side by side
  for (int w = threadIdx.x; w < (kTile / 4) * K; w += blockDim.x) {
    const int c = w / (kTile / 4), r = 4 * (w % (kTile / 4));
    const int4 tg = *reinterpret_cast<const int4*>(tile_tgt + (int64_t)tile * kTile + r);
    if ((tg.x & tg.y & tg.z & tg.w) < 0) continue;  // all four rows empty
    const float* pp = part + ((int64_t)lq * Kp + c) * kTile + r;
    float4 sum = make_float4(0.f, 0.f, 0.f, 0.f), comp = sum;
    auto kahan = [](float& sm, float& cm, float v) {
      const float y = v - cm;
      const float tt = sm + y;
      cm = (tt - sm) - y;
      sm = tt;
    };
    for (int b = c0; b < c1; b += 8) {
      float4 v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k)
        v[k] = b + k < c1 ? __ldcs(reinterpret_cast<const float4*>(pp + (int64_t)(b + k) * cstride))
                          : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (b + k >= c1) break;
        kahan(sum.x, comp.x, v[k].x);
        kahan(sum.y, comp.y, v[k].y);
        kahan(sum.z, comp.z, v[k].z);
        kahan(sum.w, comp.w, v[k].w);
      }
    }
    if (tg.x >= 0) L[(int64_t)tg.x * Kp + c] = sum.x;
    if (tg.y >= 0) L[(int64_t)tg.y * Kp + c] = sum.y;
    if (tg.z >= 0) L[(int64_t)tg.z * Kp + c] = sum.z;
    if (tg.w >= 0) L[(int64_t)tg.w * Kp + c] = sum.w;
  }
}

// hi = tf32(x) and lo = tf32(x - hi) (both rounded to nearest), for the
// multipoles.
__global__ void k_split_tf32(const float* __restrict__ x, int64_t n, float* __restrict__ hi, float* __restrict__ lo) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = x[i];
  uint32_t hb;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(v));
  const float h = __uint_as_float(hb);
  hi[i] = h;
  uint32_t lb;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lb) : "f"(v - h));
  lo[i] = __uint_as_float(lb);
}

// L rows of one tile = compensated (Kahan) sum of its chunks' partials, in
// chunk order.  Thread per (coefficient, row), rows fastest (the partials
// are column-major).
__global__ void k_m2l_reduce(const int32_t* __restrict__ tile_tgt, const int32_t* __restrict__ tile_cptr,
                             const float* __restrict__ part, int K, int Kp, float* __restrict__ L) {
  const int tile = blockIdx.x;
  const int c0 = tile_cptr[tile], c1 = tile_cptr[tile + 1];
  for (int w = threadIdx.x; w < kTile * K; w += blockDim.x) {
    const int c = w / kTile, r = w % kTile;
    const int tgt = tile_tgt[(int64_t)tile * kTile + r];
    if (tgt < 0) continue;
    float sum = 0.f, comp = 0.f;
    for (int ch = c0; ch < c1; ++ch) {
      const float y = __ldcs(part + ((int64_t)ch * Kp + c) * kTile + r) - comp;
      const float tt = sum + y;
      comp = (tt - sum) - y;
      sum = tt;
    }
    L[(int64_t)tgt * Kp + c] = sum;
  }
}

}  // namespace

int m2l_tc_stages(int Kp) {
  const int stage_bytes = 2 * kStageA + 2 * Kp * kRowB;
  int s = (200 * 1024) / stage_bytes;  // two stages still fit at Kp = 256
  return s < 2 ? 2 : (s > kMaxStages ? kMaxStages : s);
}

void launch_split_tf32(fmm_tree* t, cudaStream_t s) {
  const int64_t n = (int64_t)t->ncell * t->Kp;
  k_split_tf32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const float*)t->M, n, t->M_lo + n, t->M_lo);
  GB_LAUNCH("k_split_tf32");
}

// Quad engine source-row stages: what fits next to the two operator stages.
int m2l_tc4_astages(int Kp) {
  const int s = (200 * 1024 - 4 * Kp * kRowB) / (2 * kStageA);
  return s < 2 ? 2 : (s > kMaxAStages ? kMaxAStages : s);
}

void launch_m2l_tcgen05(fmm_tree* t, cudaStream_t s) {
  if (t->ntile == 0) return;
  const int Kp = t->Kp;
  if (t->m2l_quad) {
    const int na = m2l_tc4_astages(Kp);
    const size_t smem = (size_t)4 * Kp * kRowB + (size_t)na * 2 * kStageA + 1024;
    GB_CK(cudaFuncSetAttribute(k_m2l_tc4, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t n = (int64_t)t->ncell * Kp;
    k_m2l_tc4<<<t->nchunk, kThreadsTC, smem, s>>>(t->m2l_ops_map[0], t->m2l_ops_map[1], t->m2l_chunks, t->quad_class,
                                                  t->quad_entry, t->entry_src, t->M_lo + n, t->M_lo, Kp, (t->K + 7) & ~7, na,
                                                  t->m2l_part, t->dev_err);
    GB_LAUNCH("k_m2l_tc4");
    k_m2l_reduce4<<<t->ntile, 512, 0, s>>>(t->tile_tgt, t->tile_cptr, t->m2l_part, t->K, Kp, (float*)t->L);
    GB_LAUNCH("k_m2l_reduce4");
    return;
  }
  const int nstage = m2l_tc_stages(Kp);
  const size_t smem = (size_t)nstage * (2 * kStageA + 2 * Kp * kRowB) + 1024;
  // the dynamic size this launch needs (static + dynamic must stay within the
  // 227 KB per-block limit)
  int cols = 32;
  while (cols < Kp) cols <<= 1;
  const int64_t n = (int64_t)t->ncell * Kp;
  if (2 * cols <= 512 && m2l_fold_enabled()) {
    GB_CK(cudaFuncSetAttribute(k_m2l_tc_fold, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_m2l_tc_fold<<<t->nchunk, kThreadsFold, smem, s>>>(t->m2l_ops_map[0], t->m2l_ops_map[1], t->m2l_chunks,
                                                        t->entry_class, t->entry_src, t->M_lo + n, t->M_lo, Kp,
                                                        nstage, cols, t->m2l_part, t->dev_err);
    GB_LAUNCH("k_m2l_tc_fold");
  } else {
    GB_CK(cudaFuncSetAttribute(k_m2l_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_m2l_tc<<<t->nchunk, kThreadsTC, smem, s>>>(t->m2l_ops_map[0], t->m2l_ops_map[1], t->m2l_chunks,
                                                 t->entry_class, t->entry_src, t->M_lo + n, t->M_lo, Kp, nstage, cols,
                                                 t->m2l_part, t->dev_err);
    GB_LAUNCH("k_m2l_tc");
  }
  k_m2l_reduce<<<t->ntile, 256, 0, s>>>(t->tile_tgt, t->tile_cptr, t->m2l_part, t->K, Kp, (float*)t->L);
  GB_LAUNCH("k_m2l_reduce");
}

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver, found through the runtime (the
// library does not link libcuda)
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    GB_CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p) fail(FMM_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// The operators as one fp32 row-major [nclass * Kp][Kp] matrix; boxes of
// 32 columns x Kp rows (one k-block of one operator), 128-byte swizzle.
void make_ops_map(CUtensorMap* map, const float* ptr, int64_t rows, int Kp) {
  const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)Kp * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kKB, (cuuint32_t)Kp};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode_tiled()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(ptr), dims, strides,
                                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(FMM_ERR_CUDA, "cuTensorMapEncodeTiled (M2L operators) failed");
}

}  // namespace

// Chunks of at most `per` consecutive entries of every tile (host: the entry
// ranges of the tiles are read back once at build time), the partial buffer
// and the split multipole copies.  Partial slots are numbered tile by tile
// (chunk .w); the launch order is chunk-within-tile major, so the CTAs that
// run at the same time work on the same stretch of every tile's class list
// and share the translation operators in L2.
namespace {

// Quad plan on the device through a dense (quad, class) table: marking the
// pairs present and scanning the marks numbers the quad entries in (quad,
// class) order, which is the merge of the four tiles' sorted class lists.
__device__ __forceinline__ int tile_of_entry(const int32_t* __restrict__ tile_eptr, int ntile, int e) {
  int lo = 0, hi = ntile;  // last tile whose first entry is <= e
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (tile_eptr[mid] <= e) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void k_quad_mark(const int32_t* __restrict__ tile_eptr, int ntile, const int32_t* __restrict__ entry_class,
                            int nentry, int nclass, int64_t* __restrict__ mark) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nentry) return;
  const int tile = tile_of_entry(tile_eptr, ntile, e);
  mark[(int64_t)(tile / kQuad) * nclass + entry_class[e]] = 1;
}

__global__ void k_quad_fill(const int32_t* __restrict__ tile_eptr, int ntile, const int32_t* __restrict__ entry_class,
                            int nentry, int nclass, const int64_t* __restrict__ qid, int32_t* __restrict__ qcls,
                            int32_t* __restrict__ qent) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nentry) return;
  const int tile = tile_of_entry(tile_eptr, ntile, e);
  const int c = entry_class[e];
  const int64_t j = qid[(int64_t)(tile / kQuad) * nclass + c];
  qent[4 * j + (tile % kQuad)] = e;
  qcls[j] = c;  // the entries of one quad entry all write the same class
}

// Chunk list of a plan from the entry pointers of its groups (quads, or
// tiles for the single-tile engine): chunks of at most `per` entries, chunk
// j of every group before chunk j + 1 of any (the operators of a class are
// then still in L2 when the next group asks for them), and each group's
// first partial slot.  k_chunk_rounds (one block): each group's chunk count
// nc and first slot, and the first position of round j, the rounds holding
// #{groups with nc > j} chunks each (nround >= the largest nc, counts in
// hist[0 .. nround], zeroed).  k_chunk_place: thread g places its chunks,
// its position within a round taken by an atomic counter; the order within
// a round changes nothing but which block runs a chunk (each chunk writes
// its own partial slot).
__global__ void __launch_bounds__(1024) k_chunk_rounds(const int32_t* __restrict__ gptr, int ngroup, int per,
                                                       int nround, int32_t* __restrict__ cptr,
                                                       int* __restrict__ hist, int* __restrict__ round_at,
                                                       long long* __restrict__ nchunk) {
  __shared__ int wsum[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int run = 0;
  for (int g0 = 0; g0 < ngroup; g0 += blockDim.x) {
    const int g = g0 + threadIdx.x;
    const int nc = g < ngroup ? (gptr[g + 1] - gptr[g] + per - 1) / per : 0;
    if (nc) atomicAdd(&hist[min(nc, nround)], 1);
    int inc = nc;
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += u;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    int before = 0, all = 0;
    for (int q = 0; q < nw; ++q) {
      before += q < w ? wsum[q] : 0;
      all += wsum[q];
    }
    __syncthreads();
    if (g < ngroup) cptr[g] = run + before + inc - nc;
    run += all;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    cptr[ngroup] = run;
    *nchunk = run;
    // groups with nc > j = sum of hist[c], c > j
    int above = 0;
    for (int c = 1; c <= nround; ++c) above += hist[c];
    int at = 0;
    for (int j = 0; j < nround; ++j) {
      round_at[j] = at;
      at += above;
      above -= hist[j + 1];
    }
  }
}

__global__ void k_chunk_place(const int32_t* __restrict__ gptr, int ngroup, int per, const int32_t* __restrict__ cptr,
                              const int* __restrict__ round_at, int* __restrict__ round_fill,
                              int4* __restrict__ chunks) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ngroup) return;
  const int nc = (gptr[g + 1] - gptr[g] + per - 1) / per;
  for (int j = 0; j < nc; ++j) {
    const int e = gptr[g] + j * per;
    chunks[round_at[j] + atomicAdd(&round_fill[j], 1)] = make_int4(g, e, min(e + per, gptr[g + 1]), cptr[g] + j);
  }
}

// The quad ptr from the scanned (quad, class) table; its total is on the device.
__global__ void k_quad_ptr_dev(const int64_t* __restrict__ qid, int nquad, int nclass,
                               const int64_t* __restrict__ total, int32_t* __restrict__ qptr) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q > nquad) return;
  qptr[q] = (int32_t)(q < nquad ? qid[(int64_t)q * nclass] : *total);
}

}  // namespace

// The chunk list on the device from group entry pointers; the chunk count is
// read back with the build's last read-back (t->d_tail[3]), and the partial
// buffer is allocated then (finish_m2l_chunks).
void build_chunk_list(fmm_tree* t, const int32_t* d_gptr, int ngroup, int per, int64_t max_chunks) {
  Arena& a = t->arena;
  cudaStream_t s = t->stream;
  t->m2l_chunks = alloc_n<int4>(a, std::max<int64_t>(1, max_chunks));
  t->tile_cptr = alloc_n<int32_t>(a, ngroup + 1);
  // a group holds at most nclass entries (one per class)
  const int nround = (t->nclass + per - 1) / per + 1;
  int* work = alloc_n<int>(a, 3 * (size_t)nround + 1);  // hist[0 .. nround], round_at, round_fill
  GB_CK(cudaMemsetAsync(work, 0, sizeof(int) * (3 * (size_t)nround + 1), s));
  int *hist = work, *round_at = work + nround + 1, *round_fill = round_at + nround;
  k_chunk_rounds<<<1, 1024, 0, s>>>(d_gptr, ngroup, per, nround, t->tile_cptr, hist, round_at, t->d_tail + 3);
  GB_LAUNCH("k_chunk_rounds");
  if (ngroup > 0) {
    k_chunk_place<<<(unsigned)((ngroup + 255) / 256), 256, 0, s>>>(d_gptr, ngroup, per, t->tile_cptr, round_at,
                                                                  round_fill, t->m2l_chunks);
    GB_LAUNCH("k_chunk_place");
  }
  a.release(work);
}

// Quad plan: the class lists of tiles 4q .. 4q + 3 (each sorted by class)
// merged into quad entries, cut into chunks of at most `per` quad entries.
void build_m2l_quads(fmm_tree* t, int per) {
  Arena& a = t->arena;
  cudaStream_t s = t->stream;
  const int nquad = (t->ntile + kQuad - 1) / kQuad;
  const int64_t nk = (int64_t)nquad * t->nclass;
  t->m2l_quad = true;
  t->m2l_part_per_chunk = (int64_t)kQuad * kTile * t->Kp;
  // a quad entry holds at least one tile entry, and a quad's chunks are at
  // most its entries / per + 1
  const int64_t max_chunks = (t->nentry + per - 1) / per + nquad;
  int32_t* d_qptr = alloc_n<int32_t>(a, nquad + 1);
  if (nk > 0 && nk <= (1ll << 22) && t->nentry > 0) {
    int64_t* qid = alloc_n<int64_t>(a, nk);
    int64_t* nq = alloc_n<int64_t>(a, 1);
    GB_CK(cudaMemsetAsync(qid, 0, sizeof(int64_t) * nk, s));
    const unsigned nb = (unsigned)((t->nentry + 255) / 256);
    k_quad_mark<<<nb, 256, 0, s>>>(t->tile_eptr, t->ntile, t->entry_class, (int)t->nentry, t->nclass, qid);
    GB_LAUNCH("k_quad_mark");
    scan_exclusive_i64_dev(a, qid, nk, nq, s);
    t->quad_class = alloc_n<int32_t>(a, t->nentry);
    t->quad_entry = alloc_n<int4>(a, t->nentry);
    GB_CK(cudaMemsetAsync(t->quad_entry, 0xff, sizeof(int4) * t->nentry, s));  // -1: no entry of that tile
    k_quad_fill<<<nb, 256, 0, s>>>(t->tile_eptr, t->ntile, t->entry_class, (int)t->nentry, t->nclass, qid,
                                   t->quad_class, reinterpret_cast<int32_t*>(t->quad_entry));
    GB_LAUNCH("k_quad_fill");
    k_quad_ptr_dev<<<(unsigned)((nquad + 256) / 256), 256, 0, s>>>(qid, nquad, t->nclass, nq, d_qptr);
    GB_LAUNCH("k_quad_ptr_dev");
    build_chunk_list(t, d_qptr, nquad, per, max_chunks);
    a.release(nq);
    a.release(qid);
    a.release(d_qptr);
    return;
  }
  // a class table too large for the device marks: the quad entries merged on
  // the host from the tiles' class lists
  std::vector<int32_t> eptr(t->ntile + 1), ecls(t->nentry);
  GB_CK(cudaMemcpyAsync(eptr.data(), t->tile_eptr, sizeof(int32_t) * (t->ntile + 1), cudaMemcpyDeviceToHost, s));
  if (t->nentry)
    GB_CK(cudaMemcpyAsync(ecls.data(), t->entry_class, sizeof(int32_t) * t->nentry, cudaMemcpyDeviceToHost, s));
  host_sync(a, s);
  std::vector<int32_t> qcls, qptr(nquad + 1, 0);
  std::vector<int4> qent;
  qcls.reserve(t->nentry);
  qent.reserve(t->nentry);
  for (int q = 0; q < nquad; ++q) {
    int p[kQuad], end[kQuad];
    for (int l = 0; l < kQuad; ++l) {
      const int tile = q * kQuad + l;
      p[l] = tile < t->ntile ? eptr[tile] : 0;
      end[l] = tile < t->ntile ? eptr[tile + 1] : 0;
    }
    for (;;) {
      int c = -1;
      for (int l = 0; l < kQuad; ++l)
        if (p[l] < end[l] && (c < 0 || ecls[p[l]] < c)) c = ecls[p[l]];
      if (c < 0) break;
      int e[kQuad];
      for (int l = 0; l < kQuad; ++l) e[l] = (p[l] < end[l] && ecls[p[l]] == c) ? p[l]++ : -1;
      qcls.push_back(c);
      qent.push_back(make_int4(e[0], e[1], e[2], e[3]));
    }
    qptr[q + 1] = (int32_t)qcls.size();
  }
  t->quad_class = alloc_n<int32_t>(a, qcls.size());
  t->quad_entry = alloc_n<int4>(a, qent.size());
  if (!qcls.empty()) {
    GB_CK(cudaMemcpyAsync(t->quad_class, qcls.data(), sizeof(int32_t) * qcls.size(), cudaMemcpyHostToDevice, s));
    GB_CK(cudaMemcpyAsync(t->quad_entry, qent.data(), sizeof(int4) * qent.size(), cudaMemcpyHostToDevice, s));
  }
  // a copy from pageable memory has read its source when it returns
  GB_CK(cudaMemcpyAsync(d_qptr, qptr.data(), sizeof(int32_t) * (nquad + 1), cudaMemcpyHostToDevice, s));
  build_chunk_list(t, d_qptr, nquad, per, max_chunks);
  a.release(d_qptr);
}

void build_m2l_chunks(fmm_tree* t, int per) {
  Arena& a = t->arena;
  t->M_lo = alloc_n<float>(a, 2 * (size_t)t->ncell * t->Kp);
  if (t->nclass > 0) {
    const int64_t rows = (int64_t)t->nclass * t->Kp;
    make_ops_map(&t->m2l_ops_map[0], (const float*)t->m2l_ops, rows, t->Kp);
    make_ops_map(&t->m2l_ops_map[1], t->m2l_ops_lo, rows, t->Kp);
  }
  if (t->Kp <= kQuadMaxKp && !m2l_single_tile_forced()) {
    build_m2l_quads(t, per);
    return;
  }
  t->m2l_part_per_chunk = (int64_t)kTile * t->Kp;
  build_chunk_list(t, t->tile_eptr, t->ntile, per, (t->nentry + per - 1) / per + t->ntile);
}

// After the build's last read-back: the chunk count and the partial buffer.
void finish_m2l_chunks(fmm_tree* t, int64_t nchunk) {
  t->nchunk = (int)nchunk;
  t->m2l_part = alloc_n<float>(t->arena, (size_t)std::max<int64_t>(1, nchunk) * t->m2l_part_per_chunk);
}

}  // namespace gbfmm

// host out[16]: the quad engine's trace counters (see g_m2l_trace), read and
// cleared.  Returns 1 in a trace build, 0 (and zeros) otherwise.
extern "C" int fmm_debug_m2l_trace(int64_t* out) {
  if (!out) return FMM_ERR_ARG;
  for (int k = 0; k < 16; ++k) out[k] = 0;
#ifdef GBFMM_M2L_TRACE
  unsigned long long h[16] = {0};
  if (cudaMemcpyFromSymbol(h, gbfmm::g_m2l_trace, sizeof(h)) != cudaSuccess) {
    cudaGetLastError();
    return FMM_ERR_CUDA;
  }
  const unsigned long long z[16] = {0};
  cudaMemcpyToSymbol(gbfmm::g_m2l_trace, z, sizeof(z));
  for (int k = 0; k < 16; ++k) out[k] = (int64_t)h[k];
  return 1;
#else
  return FMM_OK;
#endif
}
