// common.cuh -- internal declarations shared by the gbfmm CUDA sources.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "gbfmm.h"

namespace gbfmm {

constexpr int kMaxLevel = 21;   // 63-bit Morton keys, 3 bits per level (Sec. II.B)
constexpr int kMaxP = 16;       // expansion terms supported (K = p*p <= 256)
constexpr int kTile = 128;      // targets per M2L tile (rows of one MMA / one CTA)
constexpr int kM2LChunk = 16;   // entries accumulated per TMEM partial (tensor-core M2L)

// Bits of a tree's device error word (fmm_tree::dev_err), set by kernels
// whose bounded waits gave up; the word is sticky for the tree's life.
constexpr int kErrWait = 1;   // an evaluation kernel gave up on a copy or MMA: that pass is invalid
constexpr int kErrScan = 2;   // a device scan's look-back gave up: the build is invalid
constexpr int kErrDrain = 4;  // a block ended while a copy or MMA it issued had not been seen to complete
constexpr int kErrGrid = 8;   // a grid barrier of a cooperative build kernel gave up: the build is invalid

struct Error {
  int code;
  std::string what;
};

[[noreturn]] void fail(int code, const char* what);
extern thread_local std::string g_last_error;
void check_cuda(cudaError_t e, const char* what);
void count_launch();
#define GB_CK(call) ::gbfmm::check_cuda((call), #call)
// after every kernel launch: count it and surface a launch error
#define GB_LAUNCH(what) (::gbfmm::count_launch(), ::gbfmm::check_cuda(cudaGetLastError(), what))

// Stream-ordered device memory through the caller's allocator or the
// library's memory pool.  Every allocation of a tree is recorded for release.
cudaMemPool_t library_pool();
struct Arena {
  fmm_allocator user{};
  bool has_user = false;
  cudaStream_t stream = nullptr;
  int* err = nullptr;  // the owning tree's device error word (kErr* bits), set before any scan
  int nsync = 0;       // host synchronisations of the stream (host_sync)
  std::vector<void*> live;
  void* alloc(size_t bytes);
  void release(void* p);
  void release_all();
  size_t bytes = 0;
};

template <class T>
T* alloc_n(Arena& a, size_t n) {
  return static_cast<T*>(a.alloc(sizeof(T) * (n ? n : 1)));
}

// ---------------------------------------------------------------- device prims
// Exclusive scans of n nonnegative int64 values in place.  A scan whose
// bounded look-back wait gave up sets kErrScan in *a.err; kernels that
// consume a scan's offsets before the host has looked at that word skip
// their work once it is set (they take the error word as an argument).
void scan_exclusive_i64(Arena& a, int64_t* d, int64_t n, cudaStream_t s);
// the total is left in device memory (no host synchronisation)
void scan_exclusive_i64_dev(Arena& a, int64_t* d, int64_t n, int64_t* total_dev, cudaStream_t s);
// returns the total: synchronises the stream, reads the total and the error
// word, and fails with FMM_ERR_TIMEOUT if kErrScan is set
int64_t scan_exclusive_i64_total(Arena& a, int64_t* d, int64_t n, cudaStream_t s);
// host: waits for the stream and counts the wait in a.nsync (every host
// synchronisation of a build goes through it)
void host_sync(Arena& a, cudaStream_t s);
// host: fails with FMM_ERR_TIMEOUT if kErrScan is set in the error word
// (synchronises the stream first)
void check_scan_error(Arena& a, cudaStream_t s);

// LSD radix sort of (key, value) pairs on bits [0, bits) of the key; stable.
// keys/vals are replaced by the sorted arrays (ping-pong buffers from the arena).
void radix_sort_pairs(Arena& a, uint64_t*& keys, int32_t*& vals, int64_t n, int bits,
                      cudaStream_t s);
void radix_sort_keys(Arena& a, uint64_t*& keys, int64_t n, int bits, cudaStream_t s);

// Root cube of the bounding box (Sec. II.C "local bounding box").
struct RootBox {
  double lo[3], hi[3], centre[3], H, corner[3];
  int nonfinite;
};

// ------------------------------------------------------------------- the tree
// Array sizes of a tree, passed to the evaluation kernels (bounds of the
// self-checking build) and the record of the first violation.
struct Lim {
  long long N, ncell, nleaf, Kp, ntile, nentry, nclass, nranges;
  unsigned long long* rec;
};

struct Cells {
  int32_t *level = nullptr, *ix = nullptr, *iy = nullptr, *iz = nullptr;
  int32_t *bbeg = nullptr, *bend = nullptr, *cbeg = nullptr, *nch = nullptr, *parent = nullptr;
};

}  // namespace gbfmm

struct fmm_tree {
  int precision = 32;  // 32 or 64 (bits of the working real type)
  int64_t N = 0;
  int p = 0, K = 0, Kp = 0, ncrit = 0;
  double theta = 0.0;
  uint32_t flags = 0;
  gbfmm::Arena arena;
  cudaStream_t stream = nullptr;  // build stream (workspace is ordered on it)

  gbfmm::RootBox root{};
  double* d_root = nullptr;  // lo3 hi3 centre3 H corner3

  void* bodies = nullptr;    // sorted (x, y, z, q) as float4 / double4
  void* work = nullptr;      // sorted bodies with the charges of the current pass
  uint64_t* keys = nullptr;  // sorted keys
  int32_t* perm = nullptr;   // sorted position -> input index

  int ncell = 0, nleaf = 0, nlevel = 0;
  std::vector<int> level_begin;  // host: first cell of each level, + end
  gbfmm::Cells c;
  int32_t* leaves = nullptr;  // leaf cell ids in cell order
  int32_t* leaf_of_cell = nullptr;  // cell -> leaf index or -1
  // FMM_FLAG_FITTED_CENTRES: integer centres (3 per cell, units H / 2^21),
  // expansion centres (3 doubles per cell) and their float pairs (hi[3],
  // lo[3] per cell), and the M2L list as CSR by target (sources in order)
  int32_t* fit_c = nullptr;
  double* fit_cen = nullptr;
  float* fit_cenf = nullptr;
  int32_t* m2l_ptr = nullptr;
  int32_t* m2l_csr_src = nullptr;
  int fit_ntgt = 0;                 // cells with M2L sources, and their ids
  int32_t* fit_tgts = nullptr;

  int64_t n_p2p = 0, n_m2l = 0, n_p2p_ranges = 0, p2p_body_pairs = 0;
  int32_t *p2p_tgt = nullptr, *p2p_src = nullptr, *m2l_tgt = nullptr, *m2l_src = nullptr;
  int32_t* m2l_has = nullptr;             // per cell: takes M2L (traversal, for the plan)
  uint32_t* m2l_off = nullptr;            // per M2L entry: packed class offset (traversal, for the plan)
  long long* d_tail = nullptr;            // read back at the end of the build: P2P ranges, body pairs + N,
                                          // operator range flag, M2L chunks
  int64_t m2l_part_per_chunk = 0;         // floats of one chunk's partial sums
  int64_t m2l_ntgt = 0;                   // cells that take M2L (from the traversal)
  unsigned long long m2l_maxd_host = 0;   // largest M2L class offset component (from the traversal)
  unsigned long long* m2l_maxd = nullptr;  // largest M2L class offset component (traversal, for the plan)
  int32_t* p2p_rptr = nullptr;  // per leaf: ranges [rptr[l], rptr[l+1])
  int2* p2p_ranges = nullptr;   // (begin, end) sorted body ranges, self excluded
  int64_t n_p2p_upairs = 0;     // mutual interaction: unordered leaf pairs (cells a < b)
  int2* p2p_upairs = nullptr;

  // M2L engine: targets tiled kTile at a time, per tile one entry per
  // translation operator with the source of each tile row (or -1).
  int nclass = 0, ntile = 0;
  int64_t nentry = 0;
  int32_t* class_desc = nullptr;   // 4 per class: level_src - level_tgt, dx, dy, dz
  int32_t* tile_tgt = nullptr;     // ntile x kTile target cells (-1 = empty row)
  int32_t* tile_eptr = nullptr;    // ntile + 1
  int32_t* entry_class = nullptr;  // nentry
  int32_t* entry_src = nullptr;    // nentry x kTile
  void* m2l_ops = nullptr;         // nclass x Kp x Kp (out-major), working precision
  float* m2l_ops_lo = nullptr;     // low parts for the 3xTF32 engine
  CUtensorMap m2l_ops_map[2] = {}; // TMA maps of the operator hi / lo parts (tensor-core engine)
  int m2l_engine = 0;
  void* m2m_ops = nullptr;  // 8 x Kp x Kp
  void* l2l_ops = nullptr;  // 8 x Kp x Kp

  void* M = nullptr;  // ncell x Kp
  void* L = nullptr;  // ncell x Kp
  float* M_lo = nullptr;  // split copy of M for the 3xTF32 engine (lo | hi)
  int nchunk = 0;                  // M2L work units of the tensor-core engine
  int4* m2l_chunks = nullptr;      // single-tile engine: (tile, first entry, end entry, partial slot);
                                   // quad engine: (quad, first quad entry, end quad entry, chunk)
  int32_t* tile_cptr = nullptr;    // single-tile: partial slots of tile t [cptr[t], cptr[t+1]);
                                   // quad: chunks of quad q [cptr[q], cptr[q+1])
  float* m2l_part = nullptr;       // partial local expansions, Kp x kTile each
  bool m2l_quad = false;           // four tiles per CTA sharing each operator k-block
  int32_t* quad_class = nullptr;   // per quad entry: the class
  int4* quad_entry = nullptr;      // per quad entry: the entry of each of the quad's tiles (-1: none)
  void* near = nullptr;   // N x 4 (phi, grad) sorted, P2P part
  int4* p2p_items = nullptr;       // single precision: near-field work items (t0, nt, s, e), largest first
  int2* p2p_item_rng = nullptr;    //   and their neighbour ranges [r0, r1)
  long long* p2p_nitem = nullptr;  //   item count, then the count of per-block items (device)
  int build_syncs = 0;              // host synchronisations of fmm_build
  int64_t p2p_nbig_host = 0;       //   items of the per-block kernel (the first ones), read back
  int64_t p2p_nitem_max = 0;       //   bound on it (array size)
  int64_t p2p_nitem_host = 0;      //   item count, read back at the end of the build
  void* near_src = nullptr;  // single precision: the P2P sources, bodies 2m and 2m + 1 in 32-byte pair m
  void* grad_q = nullptr; // N x 4 (phi, grad) sorted, of the last evaluate
  void* q_last = nullptr; // N sorted charges of the last evaluate
  int evaluations = 0;

  unsigned long long* check_rec = nullptr;  // self-check record (checked build)
  int* dev_err = nullptr;  // kErr* bits set by kernels whose bounded waits gave up (sticky)
  cudaEvent_t pass_done = nullptr;  // recorded at the end of every evaluate / backward
  gbfmm::Lim lim{};
  cudaStream_t side = nullptr;  // P2P runs here (lowest priority), concurrently with the far field
  cudaStream_t far = nullptr;   // the far field runs here (highest priority)
  cudaEvent_t fork = nullptr, join = nullptr, fork_near = nullptr, join_far = nullptr;
  cudaEvent_t ev[2 * FMM_PH_COUNT] = {};
  float ms[FMM_PH_COUNT] = {};
};

namespace gbfmm {

// Tree construction (tree.cu)
void build_tree(fmm_tree* t, const void* xyzq, bool f64);
// Traversal and lists (traverse.cu)
void build_lists(fmm_tree* t);
int bits_for(int64_t v);
void sort_pairs_copy(Arena& a, const int32_t* tgt, const int32_t* src, int64_t n, int ncell, int32_t* out_tgt,
                     int32_t* out_src, cudaStream_t s);
// M2L tiles and operator tables (ops.cu)
void build_m2l_plan(fmm_tree* t);
void build_operators(fmm_tree* t);
// Evaluation passes (fmm.cu)
void evaluate_pass(fmm_tree* t, const void* q_input, void* pot, void* force, cudaStream_t s,
                   bool for_backward_w, const void* w, void* dq, void* dx);

}  // namespace gbfmm
