// prims.cu -- error handling, workspace arena, device scan and radix sort.
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>

#include "common.cuh"

namespace gbfmm {

thread_local std::string g_last_error;

void fail(int code, const char* what) {
  g_last_error = what ? what : "";
  throw Error{code, g_last_error};
}

std::atomic<long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void check_cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return;
  cudaGetLastError();  // clear a sticky launch error of this thread
  std::string msg = std::string(what ? what : "") + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  fail(e == cudaErrorMemoryAllocation ? FMM_ERR_OOM : FMM_ERR_CUDA, msg.c_str());
}

// The library's stream-ordered memory pool on the current device.  Unlike
// the device's default pool (release threshold 0), it keeps up to
// kPoolKeepBytes of freed memory mapped for reuse across synchronisations,
// so the many short-lived buffers of fmm_build and repeated builds do not
// map and unmap physical memory every time.
constexpr uint64_t kPoolKeepBytes = 16ull << 30;

cudaMemPool_t library_pool() {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  int dev = 0;
  GB_CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) return it->second;
  cudaMemPoolProps props;
  memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  GB_CK(cudaMemPoolCreate(&pool, &props));
  uint64_t keep = kPoolKeepBytes;
  GB_CK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
  pools[dev] = pool;
  return pool;
}

void* Arena::alloc(size_t n) {
  void* p = nullptr;
  if (has_user) {
    p = user.alloc(n, (fmm_stream)stream, user.ctx);
    if (!p) fail(FMM_ERR_OOM, "user allocator");
  } else {
    cudaError_t e = cudaMallocFromPoolAsync(&p, n, library_pool(), stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      fail(e == cudaErrorMemoryAllocation ? FMM_ERR_OOM : FMM_ERR_CUDA, "cudaMallocFromPoolAsync");
    }
  }
  live.push_back(p);
  bytes += n;
  return p;
}

void Arena::release(void* p) {
  if (!p) return;
  for (size_t i = 0; i < live.size(); ++i)
    if (live[i] == p) {
      live[i] = live.back();
      live.pop_back();
      break;
    }
  if (has_user) user.free(p, (fmm_stream)stream, user.ctx);
  else cudaFreeAsync(p, stream);
}

void Arena::release_all() {
  for (void* p : live) {
    if (has_user) user.free(p, (fmm_stream)stream, user.ctx);
    else cudaFreeAsync(p, stream);
  }
  live.clear();
  bytes = 0;
}

// ------------------------------------------------------------------- scan
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ int64_t block_exclusive_scan(int64_t v, int64_t* total) {
  __shared__ int64_t warp_sums[kScanThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int64_t w = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
    int64_t s = w;
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = s - w;
    if (lane == kScanThreads / 32 - 1) *total = s;
  }
  __syncthreads();
  int64_t r = warp_sums[wid] + x - v;
  __syncthreads();
  return r;
}

// In-place exclusive scan of at most one tile (a single block).
__global__ void k_scan_tile(int64_t* __restrict__ d, int64_t n, int64_t* __restrict__ total) {
  const int64_t base = (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? d[base + i] : 0;
    s += v[i];
  }
  __shared__ int64_t btotal;
  int64_t run = block_exclusive_scan(s, &btotal);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) d[base + i] = run;
    run += v[i];
  }
  if (total && threadIdx.x == 0) *total = btotal;
}

// Single-pass scan (decoupled look-back): each block takes a ticket, scans
// its tile, publishes the tile's sum, then adds the published values of the
// tiles before it, walking back (32 tiles per step, one per lane of warp 0)
// until one that already holds its inclusive prefix, and publishes its own.
// A block only waits for blocks that took their tickets earlier and never
// for later ones, so every wait ends.  The wait is bounded all the same, by
// the device clock (%globaltimer, ns): past soft_ns it sets kErrScan in *err
// (the host then fails the call with FMM_ERR_TIMEOUT) and keeps waiting, so
// that the offsets every later kernel uses stay correct; past kScanHardNs it
// gives up for good and the scan's result is not valid.  No copy is in
// flight in this kernel, so giving up is safe for the kernel itself.
//
// late_first_ns (test switch, fmm_debug_scan_fault): tile 0 publishes only
// after that delay, so the look-back of the tiles after it runs past a soft
// limit shorter than the delay.
constexpr unsigned long long kStatAgg = 1ull << 62, kStatInc = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;
constexpr long long kScanSoftNs = 50000000ll;        // 50 ms: report
constexpr long long kScanHardNs = 2000000000ll;      // 2 s: give up
constexpr long long kScanFaultSoftNs = 1000000ll;    // test switch: 1 ms soft limit,
constexpr long long kScanFaultDelayNs = 10000000ll;  //   tile 0 publishes after 10 ms

std::atomic<int> g_scan_fault{0};

__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;\n" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];\n" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return (long long)t;
}

__global__ void k_scan_onepass(int64_t* __restrict__ d, int64_t n, int64_t* __restrict__ total,
                               unsigned long long* __restrict__ state, unsigned* __restrict__ ticket,
                               int* __restrict__ err, long long soft_ns, long long late_first_ns) {
  __shared__ int s_tile;
  __shared__ int64_t s_prefix, btotal;
  if (threadIdx.x == 0) s_tile = (int)atomicAdd(ticket, 1u);
  __syncthreads();
  const int tile = s_tile;
  const int64_t base = (int64_t)tile * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t sum = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? d[base + i] : 0;
    sum += v[i];
  }
  const int64_t ex = block_exclusive_scan(sum, &btotal);
  if (threadIdx.x < 32) {
    // warp 0 looks back 32 tiles at a time: lane l reads tile j - l; the
    // window is usable once every tile up to the nearest inclusive one has
    // published (tiles before tile 0 count as an inclusive zero)
    const int lane = threadIdx.x;
    const int64_t agg = btotal;
    int64_t prefix = 0;
    if (tile == 0) {
      if (lane == 0) {
        if (late_first_ns > 0) {  // test switch only; bounded by the clock
          const long long t0 = global_ns();
          while (global_ns() - t0 < late_first_ns) __nanosleep(10000);
        }
        st_release(&state[0], kStatInc | (unsigned long long)agg);
      }
    } else {
      if (lane == 0) st_release(&state[tile], kStatAgg | (unsigned long long)agg);
      const long long t0 = global_ns();
      bool reported = false;
      for (int j = tile - 1; j >= 0;) {
        const int k = j - lane;
        const unsigned long long w = k >= 0 ? ld_acquire(&state[k]) : kStatInc;
        const unsigned long long st = w & ~kValMask;
        const unsigned inc = __ballot_sync(0xffffffffu, st == kStatInc);
        const unsigned avail = __ballot_sync(0xffffffffu, st != 0);
        const int first = inc ? __ffs(inc) - 1 : 31;
        const unsigned need = first == 31 ? 0xffffffffu : ((2u << first) - 1u);
        if ((avail & need) != need) {
          const long long waited = __shfl_sync(0xffffffffu, global_ns() - t0, 0);
          if (waited > soft_ns && !reported) {
            if (lane == 0) atomicOr(err, kErrScan);
            reported = true;
          }
          if (waited > kScanHardNs) break;  // the scan's result is not valid
          continue;
        }
        int64_t part = lane <= first ? (int64_t)(w & kValMask) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
        prefix += __shfl_sync(0xffffffffu, part, 0);
        if (inc) break;
        j -= 32;
      }
      if (lane == 0) st_release(&state[tile], kStatInc | (unsigned long long)(prefix + agg));
    }
    if (lane == 0) {
      s_prefix = prefix;
      if (total && tile == (int)gridDim.x - 1) *total = prefix + agg;
    }
  }
  __syncthreads();
  int64_t run = ex + s_prefix;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) d[base + i] = run;
    run += v[i];
  }
}

void scan_rec(Arena& a, int64_t* d, int64_t n, int64_t* total, cudaStream_t s) {
  if (!a.err) fail(FMM_ERR_CUDA, "internal: device scan without an error word");
  if (n <= 0) {
    if (total) GB_CK(cudaMemsetAsync(total, 0, sizeof(int64_t), s));
    return;
  }
  if (n <= kScanTile) {
    k_scan_tile<<<1, kScanThreads, 0, s>>>(d, n, total);
    GB_LAUNCH("k_scan_tile");
    return;
  }
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  // per-tile state words, then the ticket counter
  unsigned long long* state = alloc_n<unsigned long long>(a, nb + 1);
  GB_CK(cudaMemsetAsync(state, 0, sizeof(unsigned long long) * (nb + 1), s));
  const bool fault = g_scan_fault.load() != 0;
  k_scan_onepass<<<(unsigned)nb, kScanThreads, 0, s>>>(d, n, total, state, reinterpret_cast<unsigned*>(state + nb),
                                                       a.err, fault ? kScanFaultSoftNs : kScanSoftNs,
                                                       fault ? kScanFaultDelayNs : 0ll);
  GB_LAUNCH("k_scan_onepass");
  a.release(state);
}

}  // namespace

void host_sync(Arena& a, cudaStream_t s) {
  ++a.nsync;
  GB_CK(cudaStreamSynchronize(s));
}

void check_scan_error(Arena& a, cudaStream_t s) {
  int h = 0;
  GB_CK(cudaMemcpyAsync(&h, a.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  host_sync(a, s);
  if (h & kErrScan) fail(FMM_ERR_TIMEOUT, "a device scan's bounded look-back wait gave up");
  if (h & kErrGrid) fail(FMM_ERR_TIMEOUT, "a grid barrier of the tree build gave up");
}

void scan_exclusive_i64(Arena& a, int64_t* d, int64_t n, cudaStream_t s) {
  scan_rec(a, d, n, nullptr, s);
}

void scan_exclusive_i64_dev(Arena& a, int64_t* d, int64_t n, int64_t* total_dev, cudaStream_t s) {
  scan_rec(a, d, n, total_dev, s);
}

int64_t scan_exclusive_i64_total(Arena& a, int64_t* d, int64_t n, cudaStream_t s) {
  int64_t* tot = alloc_n<int64_t>(a, 1);
  scan_rec(a, d, n, tot, s);
  int64_t h = 0;
  GB_CK(cudaMemcpyAsync(&h, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  a.release(tot);
  check_scan_error(a, s);  // synchronises; nothing has used the result yet
  return h;
}

// ------------------------------------------------------------- radix sort
// LSD radix sort, 8-bit digits.  Pass: per-tile digit histograms (digit-major
// so that one exclusive scan gives every tile's output base per digit, in
// stable order), then a stable scatter in which each tile is consumed in
// rounds of 256 keys, ranked within the round by warp match and a per-warp
// digit count prefix.
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortRounds = 8;
constexpr int kSortTile = kSortThreads * kSortRounds;
constexpr int kRadix = 256;

__global__ void k_rs_hist(const uint64_t* __restrict__ keys, int64_t n, int shift, int ntile,
                          int64_t* __restrict__ counts) {
  __shared__ int h[kRadix];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int i = threadIdx.x; i < kSortTile; i += kSortThreads) {
    int64_t k = base + i;
    if (k < n) atomicAdd(&h[(keys[k] >> shift) & 0xff], 1);
  }
  __syncthreads();
  counts[(int64_t)threadIdx.x * ntile + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one tile.  Each key's place within the tile (its digit's
// start in the tile + its rank among the tile's keys of that digit) is found
// in rounds of 256 keys; the keys are first placed in shared memory in that
// order, then written out in order, so that neighbouring threads write
// neighbouring slots of one digit's run (coalesced).
__global__ void k_rs_scatter(const uint64_t* __restrict__ kin, const int32_t* __restrict__ vin,
                             uint64_t* __restrict__ kout, int32_t* __restrict__ vout, int64_t n,
                             int shift, int ntile, const int64_t* __restrict__ offs) {
  __shared__ int64_t gbase[kRadix];     // digit's first global slot for this tile
  __shared__ int lstart[kRadix];        // digit's first slot within the tile
  __shared__ int lrun[kRadix];          // keys of the digit placed so far
  __shared__ int wcnt[kSortThreads / 32][kRadix];
  __shared__ int wsum[kSortThreads / 32];
  __shared__ uint64_t sk[kSortTile];
  __shared__ int32_t sv[kSortTile];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, t = threadIdx.x;
  const int64_t tbase = (int64_t)blockIdx.x * kSortTile;
  const int tn = (int)(n - tbase < kSortTile ? n - tbase : kSortTile);  // keys in this tile
  {
    // this tile's count of digit t: the distance to the next (digit, tile)
    // slot of the scanned, digit-major table (the last one ends at n)
    const int64_t at = (int64_t)t * ntile + blockIdx.x;
    const int64_t start = offs[at];
    const int64_t next = at + 1 < (int64_t)kRadix * ntile ? offs[at + 1] : n;
    gbase[t] = start;
    const int c = (int)(next - start);
    // exclusive scan of the counts over the digits
    int inc = c;
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += u;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    int before = 0;
    for (int q = 0; q < wid; ++q) before += wsum[q];
    lstart[t] = before + inc - c;
    lrun[t] = 0;
  }
  for (int r = 0; r < kSortRounds; ++r) {
    for (int w = 0; w < kSortThreads / 32; ++w) wcnt[w][t] = 0;
    __syncthreads();
    const int li = r * kSortThreads + t;
    const bool valid = li < tn;
    const uint64_t key = valid ? kin[tbase + li] : 0;
    const int32_t val = (valid && vin) ? vin[tbase + li] : 0;
    const int d = valid ? (int)((key >> shift) & 0xff) : kRadix;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    const int leader = __ffs(peers) - 1;
    if (valid && lane == leader) wcnt[wid][d] = __popc(peers);
    __syncthreads();
    int rtot;
    {
      int run = 0;
      for (int w = 0; w < kSortThreads / 32; ++w) {
        const int c = wcnt[w][t];
        wcnt[w][t] = run;
        run += c;
      }
      rtot = run;
    }
    __syncthreads();
    if (valid) {
      const int pos = lstart[d] + lrun[d] + wcnt[wid][d] + rank;
      sk[pos] = key;
      sv[pos] = val;
    }
    __syncthreads();
    lrun[t] += rtot;
  }
  __syncthreads();
  for (int i = t; i < tn; i += kSortThreads) {
    const uint64_t key = sk[i];
    const int d = (int)((key >> shift) & 0xff);
    const int64_t pos = gbase[d] + (i - lstart[d]);
    kout[pos] = key;
    if (vout) vout[pos] = sv[i];
  }
}

void sort_impl(Arena& a, uint64_t*& keys, int32_t** vals, int64_t n, int bits, cudaStream_t s) {
  if (n <= 1 || bits <= 0) return;
  const int ntile = (int)((n + kSortTile - 1) / kSortTile);
  uint64_t* k2 = alloc_n<uint64_t>(a, n);
  int32_t* v2 = vals ? alloc_n<int32_t>(a, n) : nullptr;
  int64_t* counts = alloc_n<int64_t>(a, (size_t)kRadix * ntile);
  for (int shift = 0; shift < bits; shift += 8) {
    k_rs_hist<<<ntile, kSortThreads, 0, s>>>(keys, n, shift, ntile, counts);
    GB_LAUNCH("k_rs_hist");
    scan_exclusive_i64(a, counts, (int64_t)kRadix * ntile, s);
    k_rs_scatter<<<ntile, kSortThreads, 0, s>>>(keys, vals ? *vals : nullptr, k2, v2, n, shift,
                                                ntile, counts);
    GB_LAUNCH("k_rs_scatter");
    std::swap(keys, k2);
    if (vals) std::swap(*vals, v2);
  }
  a.release(counts);
  a.release(k2);
  if (v2) a.release(v2);
}

}  // namespace

void radix_sort_pairs(Arena& a, uint64_t*& keys, int32_t*& vals, int64_t n, int bits,
                      cudaStream_t s) {
  sort_impl(a, keys, &vals, n, bits, s);
}

void radix_sort_keys(Arena& a, uint64_t*& keys, int64_t n, int bits, cudaStream_t s) {
  sort_impl(a, keys, nullptr, n, bits, s);
}

}  // namespace gbfmm

extern "C" int64_t fmm_launch_count(void) { return (int64_t)gbfmm::g_launches.load(); }

extern "C" int fmm_debug_scan_fault(int on) { return gbfmm::g_scan_fault.exchange(on ? 1 : 0); }

extern "C" const char* fmm_last_error(void) { return gbfmm::g_last_error.c_str(); }
