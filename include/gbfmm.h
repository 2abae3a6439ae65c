/*
 * gbfmm.h -- C ABI of the GB300 (sm_103a) fast multipole method library
 * (libgbfmm.so).  Laplace kernel in 3-D: for N charged bodies it returns the
 * potential phi_i = sum_{j != i} q_j / |x_i - x_j| and the force per unit
 * charge -grad phi(x_i), approximated by the FMM.
 *
 * The method is the serial FMM that "Asynchronous Execution of the Fast
 * Multipole Method Using Charm++" (AbdulJabbar, Yokota, Keyes) runs on each
 * process: a local octree with Morton keys (Sec. II.B), a dual tree
 * traversal that produces the M2L and P2P interactions (Sec. II.C), the
 * upward P2M/M2M pass, M2L + P2P, and the downward L2L/L2P pass (Sec. II.A);
 * parameters P (expansion order), theta (acceptance criterion) and N_crit
 * (maximum bodies per leaf) as in Table 1 / Sec. III.A.
 *
 * Conventions
 *   - Every input and output buffer is a DEVICE pointer owned by the caller,
 *     except where an argument says "host".  Arrays are in the caller's body
 *     order ("input order"); the library never reorders the caller's data.
 *   - xyzq is N x 4, row-major (x, y, z, q) per body.
 *   - force is N x 3 row-major, force_i = -grad phi(x_i) (per unit charge;
 *     the physical force on body i is q_i * force_i).  No 1/(4 pi) factor, no
 *     softening; a body does not act on itself and bodies at the same point
 *     contribute nothing to each other.
 *   - "order p" means p terms: expansion degrees 0..p-1 (error O(theta^p)).
 *   - All calls are asynchronous and ordered on the given stream (a
 *     cudaStream_t passed as fmm_stream; NULL = the legacy default stream),
 *     except fmm_build, which waits on the stream for its counts, and the
 *     query calls marked "host".
 *   - No call aborts the process; failures return a negative code
 *     (fmm_strerror names it).  A call that fails leaves its outputs
 *     undefined but the tree handle (if any) still valid unless stated.
 *   - The tree handle owns all workspace; it is not thread-safe: calls on one
 *     handle must not run concurrently from several host threads.
 */
#ifndef GBFMM_H
#define GBFMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fmm_tree fmm_tree;
typedef void* fmm_stream; /* a cudaStream_t */

enum {
  FMM_OK = 0,
  FMM_ERR_ARG = -1,       /* invalid argument (sizes, p, theta, ncrit, null pointers) */
  FMM_ERR_NONFINITE = -2, /* a position or charge is NaN or infinite */
  FMM_ERR_OOM = -3,       /* device allocation failed */
  FMM_ERR_CUDA = -4,      /* a CUDA runtime call or kernel launch failed */
  FMM_ERR_TIMEOUT = -5,   /* a bounded device wait gave up */
  FMM_ERR_STATE = -6,     /* call out of order (e.g. backward before evaluate) */
  FMM_ERR_RANGE = -7      /* an operator coefficient is not representable in the
                             working precision (p too high for theta) */
};

/* fmm_build flags */
enum {
  FMM_FLAG_CIRCUMSCRIBED = 1u << 0, /* MAC radius = half diagonal instead of half side */
  FMM_FLAG_TIMING = 1u << 1,        /* record per-phase CUDA-event times (fmm_get_stats); the
                                       near field's events are on the stream it runs on */
  FMM_FLAG_M2L_CUDA_CORE = 1u << 2, /* single precision: M2L on CUDA cores instead of
                                       the tensor-core (3xTF32) engine */
  FMM_FLAG_SORTED_PLAN = 1u << 3,   /* number the M2L classes and (tile, class) entries by
                                       sorting the pairs, also where the dense key tables
                                       would be used; the plan is identical either way */
  FMM_FLAG_SERIAL_PHASES = 1u << 4, /* run the near field on the caller's stream after the
                                       far field instead of concurrently on a second stream
                                       (with FMM_FLAG_TIMING: each phase timed alone) */
  FMM_FLAG_MUTUAL_P2P = 1u << 5,    /* near field by mutual interaction: each unordered leaf
                                       pair visited once, both leaves updated (floating-point
                                       atomics: results are not bit-reproducible) */
  FMM_FLAG_TIGHT_MAC = 1u << 6,     /* MAC radius of a cell = the distance from its (cube)
                                       centre to its farthest body, from the 21-bit integer
                                       body coordinates (Sec. II.B's particle-fitted bound;
                                       expansion centres stay the cube centres); overrides
                                       FMM_FLAG_CIRCUMSCRIBED */
  FMM_FLAG_FITTED_CENTRES = 1u << 7 /* cells fitted to their bodies (Sec. II.B): every
                                       expansion is taken about the centre of the box of the
                                       cell's bodies (their voxel centres, 21-bit integer
                                       coordinates), and the MAC uses those centres and the
                                       distance from there to the farthest body.  Operators are
                                       no longer shared between cell pairs: M2M, L2L and M2L
                                       run per pair on CUDA cores.  The adjoint keeps the
                                       centres frozen.  Overrides FMM_FLAG_CIRCUMSCRIBED and
                                       FMM_FLAG_TIGHT_MAC */
};

/* Optional stream-ordered allocator.  NULL selects the library's memory pool
   on the current device (cudaMallocFromPoolAsync / cudaFreeAsync): it keeps up
   to 16 GiB of freed memory mapped for reuse by later calls instead of
   returning it to the driver at every synchronisation. */
typedef struct {
  void* (*alloc)(size_t bytes, fmm_stream stream, void* ctx);
  void (*free)(void* ptr, fmm_stream stream, void* ctx);
  void* ctx;
} fmm_allocator;

/* Phases timed with FMM_FLAG_TIMING (index into fmm_stats.ms). */
enum {
  FMM_PH_P2M = 0, FMM_PH_M2M, FMM_PH_M2L, FMM_PH_L2L, FMM_PH_P2P, FMM_PH_L2P,
  FMM_PH_EVAL_TOTAL, FMM_PH_BUILD_TOTAL,
  /* parts of fmm_build: cube, keys, sort and cells; dual traversal and
     P2P ranges; M2L tiles, classes and entries; operators, work chunks and
     expansion buffers */
  FMM_PH_BUILD_TREE, FMM_PH_BUILD_LISTS, FMM_PH_BUILD_PLAN, FMM_PH_BUILD_OPS,
  FMM_PH_COUNT
};

typedef struct {
  int64_t n_bodies;
  int64_t n_cells;
  int64_t n_leaves;
  int64_t n_levels;          /* levels present (root = level 0) */
  int64_t n_p2p;             /* directed leaf pairs (source, target), self pairs included */
  int64_t n_p2p_ranges;      /* merged source body ranges over all target leaves (self excluded) */
  int64_t n_p2p_body_pairs;  /* sum over P2P pairs of n_src * n_tgt, minus N (self) */
  int64_t n_m2l;             /* directed M2L pairs */
  int64_t n_m2l_classes;     /* distinct M2L translation operators */
  int64_t n_m2l_tiles;       /* target tiles of the M2L engine */
  int64_t n_m2l_slots;       /* (tile, operator) x tile-width slots processed by M2L */
  int32_t p, K, ncrit, precision_bits;
  double theta;
  uint32_t flags;
  int32_t m2l_engine;        /* 0 CUDA cores; tensor cores (tcgen05, 3xTF32): 1 one tile
                                per CTA, 2 four tiles per CTA sharing each operator;
                                3 per pair on CUDA cores (FMM_FLAG_FITTED_CENTRES) */
  int64_t workspace_bytes;   /* device bytes held by the tree */
  int32_t evaluations;       /* fmm_evaluate calls on this tree */
  int32_t device_errors;     /* bits of the tree's device error word, sticky for
                                the tree's life: 1 a bounded wait of an evaluate
                                or backward kernel gave up (that pass's outputs
                                are not valid); 4 a kernel block ended with a
                                copy or tensor-core operation it issued not seen
                                to complete (treat every output as invalid) */
  int32_t build_host_syncs;  /* times fmm_build waited for its stream (size read-backs) */
  float ms[FMM_PH_COUNT];    /* last evaluate/build phase times (FMM_FLAG_TIMING) */
} fmm_stats;

/*
 * fmm_build: bounding cube, Morton keys, sort, octree, dual tree traversal,
 * interaction lists and translation operators for one body set (Sec. II.B,
 * II.C; Table 1 parameters).
 *   xyzq   device, N x 4 float (x, y, z, q), input order.  Read only during
 *          the call; the charges become the default charges of the tree.
 *   n      number of bodies, 1 <= n <= 2^31 - 1.
 *   p      expansion order (terms), 1 <= p <= 16.
 *   theta  opening angle of the MAC  theta * |c_A - c_B| > R_A + R_B,
 *          0 < theta < 1.
 *   ncrit  a cell with more than ncrit bodies is split (up to level 21).
 *   flags  FMM_FLAG_* bits; any other bit is FMM_ERR_ARG.
 *   alloc  NULL or a stream-ordered allocator (used for all workspace).
 *   stream the stream all work is ordered on; the call synchronises it.
 *   out    host; receives the new tree handle (NULL on failure).
 * Errors: FMM_ERR_ARG, FMM_ERR_NONFINITE, FMM_ERR_OOM, FMM_ERR_CUDA,
 * FMM_ERR_RANGE, FMM_ERR_TIMEOUT (a device scan of the build waited past
 * its limit for another block: the build's blocks are not making progress
 * as they must).  On failure every byte taken from the allocator is given
 * back to it (through its free callback) before the call returns.
 */
int fmm_build(const float* xyzq, int64_t n, int p, double theta, int ncrit, uint32_t flags,
              const fmm_allocator* alloc, fmm_stream stream, fmm_tree** out);

/* Same tree from double-precision bodies; the tree then evaluates in double
 * precision (fmm_evaluate_f64 / fmm_backward_f64). */
int fmm_build_f64(const double* xyzq, int64_t n, int p, double theta, int ncrit, uint32_t flags,
                  const fmm_allocator* alloc, fmm_stream stream, fmm_tree** out);

/*
 * fmm_evaluate: P2M, M2M, M2L, L2L, L2P and P2P on the built tree
 * (Sec. II.A, II.C).
 *   q      device, N charges in input order, or NULL for the charges given
 *          to fmm_build.  Positions are always the build's.
 *   pot    device, N float, input order (required).
 *   force  device, N x 3 float, input order, or NULL.
 * The gradient of this evaluation is kept in the tree for fmm_backward.
 * Errors: FMM_ERR_ARG, FMM_ERR_STATE (tree of the other precision),
 * FMM_ERR_CUDA.
 */
int fmm_evaluate(fmm_tree* t, const float* q, float* pot, float* force, fmm_stream stream);
int fmm_evaluate_f64(fmm_tree* t, const double* q, double* pot, double* force,
                     fmm_stream stream);

/*
 * fmm_backward: adjoint of a scalar loss L with dL/dphi_i = w_i, the tree,
 * lists and expansion centres frozen.  Because the FMM operator is symmetric
 * (symmetric lists, symmetric double truncation of the even kernel 1/r),
 *   dL/dq_i = phi_w(x_i)           (an FMM pass with charges w)
 *   dL/dx_i = w_i grad phi_q(x_i) + q_i grad phi_w(x_i).
 *   w   device, N float, input order.
 *   dq  device, N float, input order.
 *   dx  device, N x 3 float, input order.
 * Requires a previous fmm_evaluate on this tree (its charges q and gradient
 * are the ones used); otherwise FMM_ERR_STATE.
 */
int fmm_backward(fmm_tree* t, const float* w, float* dq, float* dx, fmm_stream stream);
int fmm_backward_f64(fmm_tree* t, const double* w, double* dq, double* dx, fmm_stream stream);

/*
 * fmm_solve_host: one whole step through HOST buffers: copies xyzq (and w)
 * to the device, builds the tree, evaluates, runs the backward pass when w
 * is given, copies the results back and releases everything.
 *   xyzq_h  host, N x 4 float.   w_h  host, N float, or NULL (no backward).
 *   pot_h   host, N float.  force_h  host, N x 3 float, or NULL.
 *   dq_h, dx_h  host, N and N x 3 float; required when w_h is given.
 * Synchronous (returns when the host outputs are written).  Pinned host
 * memory makes the copies faster but is not required.  Returns
 * FMM_ERR_TIMEOUT (outputs not valid) when fmm_check would.
 */
int fmm_solve_host(const float* xyzq_h, const float* w_h, int64_t n, int p, double theta,
                   int ncrit, uint32_t flags, float* pot_h, float* force_h, float* dq_h,
                   float* dx_h, fmm_stream stream);

/*
 * fmm_direct_f64: reference direct sum in double precision (no tree):
 * for each listed target i, phi_i = sum_{j != i} q_j / |x_i - x_j| over all
 * n bodies (coincident bodies skipped) and force_i = -grad phi(x_i).
 * Used to report the FMM's error (accuracy, not a fast path: O(n) per target).
 *   xyzq     device, n x 4 float (the same input the tree was built from).
 *   targets  device, nt int32 input indices in [0, n); an index outside that
 *            range is not read through and gives NaN for that target.
 *   nt       0 <= nt <= 2^31 - 1.
 *   pot      device, nt double;  force  device, nt x 3 double, or NULL.
 * Errors: FMM_ERR_ARG (null pointers, n < 1, nt out of range, xyzq not
 * 16-byte aligned), FMM_ERR_CUDA.
 */
int fmm_direct_f64(const float* xyzq, int64_t n, const int32_t* targets, int64_t nt, double* pot,
                   double* force, fmm_stream stream);

/* host: number of CUDA kernels this library has launched in this process. */
int64_t fmm_launch_count(void);

/* host: statistics of the tree and of its last build/evaluate.  Waits for
 * the tree's last evaluate / backward.  Fills *out in every case and returns
 * FMM_ERR_TIMEOUT when out->device_errors is nonzero. */
int fmm_get_stats(const fmm_tree* t, fmm_stats* out);

/* host: waits for the tree's last evaluate / backward and returns
 * FMM_ERR_TIMEOUT if a bounded device wait of any pass on this tree gave up
 * (the outputs of that pass, and of any backward that uses it, are not
 * valid), else FMM_OK.  Every kernel wait is bounded so that a device fault
 * surfaces here instead of hanging the caller. */
int fmm_check(const fmm_tree* t);

/* Releases the tree and its workspace (stream-ordered on the build stream).
 * NULL is accepted. */
int fmm_destroy(fmm_tree* t);

/* host: description of the last failure in the calling thread (the failing
 * step and, for CUDA failures, the runtime's error name); empty if none. */
const char* fmm_last_error(void);

/* host: static string naming a return code. */
const char* fmm_strerror(int code);

/* ---- inspection (used by the parity tests; all device outputs, caller-owned) */

/* host out[13]: lo[3], hi[3], centre[3], H (half side of the root cube),
 * corner[3] = centre - H. */
int fmm_get_root(const fmm_tree* t, double* out);

/* keys_sorted: N uint64 Morton keys in sorted order; perm: N int32, sorted
 * position -> input index. */
int fmm_get_keys(const fmm_tree* t, uint64_t* keys_sorted, int32_t* perm, fmm_stream stream);

/* cells: 9 rows of n_cells int32, cells in breadth-first (level, Morton)
 * order: level, ix, iy, iz (integer cube coordinates at the cell's level),
 * body_begin, body_end (sorted positions), child_begin (-1 for leaves),
 * child_count, parent (-1 for the root). */
int fmm_get_cells(const fmm_tree* t, int32_t* cells, fmm_stream stream);

/* Directed interaction lists sorted by (target, source) cell:
 * p2p_tgt/p2p_src (n_p2p each), m2l_tgt/m2l_src (n_m2l each). */
int fmm_get_lists(const fmm_tree* t, int32_t* p2p_tgt, int32_t* p2p_src, int32_t* m2l_tgt,
                  int32_t* m2l_src, fmm_stream stream);

/* Expansions of the last evaluation, n_cells x K real coefficients (K = p*p,
 * float or double as the tree's precision).  Packing per degree n: index
 * n*n holds Re X_n^0, n*n + 2m - 1 and n*n + 2m hold Re and Im X_n^m
 * (m = 1..n).  Scaling: M_n^m is divided by R^n, L_n^m multiplied by
 * R^(n+1), R = half side of the cell. */
int fmm_get_expansions(const fmm_tree* t, void* M, void* L, fmm_stream stream);

/* Work plan of the M2L engine and of P2P (device outputs, caller-owned):
 *   tile_tgt     n_m2l_tiles x 128 int32: target cell of each tile row, -1 = empty
 *   tile_eptr    n_m2l_tiles + 1 int32: entries of tile t are [eptr[t], eptr[t+1])
 *   entry_class  n_entries int32: translation operator of each entry
 *   entry_src    n_entries x 128 int32: source cell per tile row, -1 = none
 *   p2p_rptr     n_leaves + 1 int32: source ranges of leaf l are [rptr[l], rptr[l+1])
 *   p2p_ranges   n_p2p_ranges x 2 int32: (body_begin, body_end), sorted positions
 * n_entries = n_m2l_slots / 128 (fmm_get_stats).  Any pointer may be NULL. */
int fmm_get_plan(const fmm_tree* t, int32_t* tile_tgt, int32_t* tile_eptr, int32_t* entry_class,
                 int32_t* entry_src, int32_t* p2p_rptr, int32_t* p2p_ranges, fmm_stream stream);

/*
 * fmm_root_keys_noalloc: the root cube and the Morton keys of fmm_build's
 * first step (same results, bit for bit), without allocating any device
 * memory.  The paper has no counterpart; this exists for callers that may
 * not allocate while they call this library: code under a fixed
 * device-memory budget or inside another framework's allocator, and code
 * that must not risk the device-wide synchronisation a cudaMalloc/cudaFree
 * can cause.  The reduction's scratch is a fixed file-scope device array
 * (about 57 KB per device, held until the process exits).
 *   xyzq       device, n x 4 float (x, y, z, q), input order.
 *   n          1 <= n <= 2^31 - 1; larger n returns FMM_ERR_ARG
 *              (fmm_last_error says why).
 *   root       device, 13 doubles, the layout of fmm_get_root.
 *   keys       device, n uint64 Morton keys in input order, or NULL.
 *   nonfinite  device int32, set to 1 if a position or charge is NaN or
 *              infinite (root and keys are then undefined), else 0; or NULL.
 * Stream-ordered and asynchronous.  The first call on a device looks up the
 * device address of the scratch array, so make that first call before any
 * stream capture.  All calls share the one scratch array: calls whose work
 * overlaps on the GPU (other streams, other host threads) race and must be
 * ordered by the caller.
 */
int fmm_root_keys_noalloc(const float* xyzq, int64_t n, double* root, uint64_t* keys, int32_t* nonfinite,
                          fmm_stream stream);

/* host, test only: on != 0 makes the first tile of every multi-tile device
 * scan publish its sum 10 ms late while the look-back's time limit drops to
 * 1 ms, so that the waiting blocks run past their limit (the scan's result
 * stays correct: they keep waiting).  fmm_build then fails with
 * FMM_ERR_TIMEOUT.  Process-wide; returns the previous setting. */
int fmm_debug_scan_fault(int on);

/* host out[16]: cycle counters of the tensor-core M2L (four-tile engine) in
 * the trace build (compiled with -DGBFMM_M2L_TRACE), summed over blocks
 * since the last read, then cleared: 0 producers waiting for a free source
 * stage, 1 producers waiting for a free operator stage, 2 the MMA thread
 * from the block's start to its loop, 3 the MMA thread from its last commit
 * to the block's end, 5 MMA waiting for an
 * operator stage, 6 MMA waiting for a source stage, 7 MMA issuing, 11 whole
 * blocks, 12 block count, 13 producers waiting for the last MMA, 14 epilogue
 * (other slots zero).  Returns 1 in a trace build, 0 (and zeros) otherwise. */
int fmm_debug_m2l_trace(int64_t* out);

/* host out[4]: record of the self-checking build (compiled with
 * -DGBFMM_CHECKED): site code and index of the first out-of-range access the
 * evaluation kernels skipped, the bound it broke, and the number of such
 * accesses.  Returns 1 in a checked build, 0 (and zeros) otherwise. */
int fmm_debug_checks(const fmm_tree* t, int64_t* out);

#ifdef __cplusplus
}
#endif

#endif /* GBFMM_H */
