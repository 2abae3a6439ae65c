// api.cu -- the C ABI (gbfmm.h): argument checks, the tree handle, and the
// order of the passes of one evaluation (Sec. II.A / II.C: upward pass
// P2M -> M2M, then M2L, downward pass L2L -> L2P; P2P alongside).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "kernels.cuh"

using namespace gbfmm;

namespace {

int to_code(const Error& e) { return e.code; }

void release_tree(fmm_tree* t) {
  if (!t) return;
  for (cudaStream_t st : {t->side, t->far})
    if (st) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
  for (cudaEvent_t e : {t->fork, t->join, t->fork_near, t->join_far, t->pass_done})
    if (e) cudaEventDestroy(e);
  for (auto& e : t->ev)
    if (e) cudaEventDestroy(e);
  t->arena.release_all();
  cudaStreamSynchronize(t->stream);
  cudaGetLastError();
  delete t;
}

template <class R>
void create_tree(fmm_tree* t, const R* xyzq) {
  const bool f64 = sizeof(R) == 8;
  t->precision = f64 ? 64 : 32;
  t->K = t->p * t->p;
  t->Kp = (t->K + 15) / 16 * 16;
  const bool fitted = (t->flags & FMM_FLAG_FITTED_CENTRES) != 0;
  t->m2l_engine = fitted ? 3 : ((!f64 && !(t->flags & FMM_FLAG_M2L_CUDA_CORE)) ? 1 : 0);
  {
    int lo = 0, hi = 0;  // numerically greatest = lowest priority
    GB_CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    GB_CK(cudaStreamCreateWithPriority(&t->side, cudaStreamNonBlocking, lo));
    GB_CK(cudaStreamCreateWithPriority(&t->far, cudaStreamNonBlocking, hi));
  }
  for (cudaEvent_t* e : {&t->fork, &t->join, &t->fork_near, &t->join_far, &t->pass_done})
    GB_CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  if (t->flags & FMM_FLAG_TIMING)
    for (auto& e : t->ev) GB_CK(cudaEventCreate(&e));
  Arena& a = t->arena;
  cudaStream_t s = t->stream;
  // the tree's device error word comes first: every device scan of the
  // build reports a wait past its limit there
  t->dev_err = alloc_n<int>(a, 1);
  GB_CK(cudaMemsetAsync(t->dev_err, 0, sizeof(int), s));
  a.err = t->dev_err;
  const bool timing = (t->flags & FMM_FLAG_TIMING) != 0;
  auto mark = [&](int ph, int end) {
    if (timing) GB_CK(cudaEventRecord(t->ev[2 * ph + end], s));
  };
  mark(FMM_PH_BUILD_TOTAL, 0);
  mark(FMM_PH_BUILD_TREE, 0);
  build_tree(t, xyzq, f64);
  mark(FMM_PH_BUILD_TREE, 1);
  mark(FMM_PH_BUILD_LISTS, 0);
  build_lists(t);
  if (!f64) build_p2p_items(t);
  mark(FMM_PH_BUILD_LISTS, 1);
  mark(FMM_PH_BUILD_PLAN, 0);
  if (fitted) {
    // fitted centres: no shared operators; the centres and the M2L list by
    // target instead of the plan
    t->tile_eptr = alloc_n<int32_t>(a, 1);
    GB_CK(cudaMemsetAsync(t->tile_eptr, 0, sizeof(int32_t), s));
    build_fitted(t);
  } else {
    build_m2l_plan(t);
  }
  a.release(t->m2l_has);
  a.release(t->m2l_maxd);
  a.release(t->m2l_off);
  t->m2l_has = nullptr;
  t->m2l_maxd = nullptr;
  t->m2l_off = nullptr;
  mark(FMM_PH_BUILD_PLAN, 1);
  mark(FMM_PH_BUILD_OPS, 0);
  if (!fitted) build_operators(t);
  const size_t rs = sizeof(R);
  t->M = a.alloc(rs * (size_t)t->ncell * t->Kp);
  t->L = a.alloc(rs * (size_t)t->ncell * t->Kp);
  GB_CK(cudaMemsetAsync(t->M, 0, rs * (size_t)t->ncell * t->Kp, s));
  t->near = a.alloc(rs * 4 * (size_t)t->N);
  if (!f64) t->near_src = a.alloc(32 * (size_t)((t->N + 1) / 2));
  t->grad_q = a.alloc(rs * 4 * (size_t)t->N);
  t->q_last = a.alloc(rs * (size_t)t->N);
  if (t->m2l_engine == 1) {
    int per = kM2LChunk;
    if (const char* env = getenv("GBFMM_M2L_CHUNK")) per = std::max(1, atoi(env));  // tuning knob
    build_m2l_chunks(t, per);
  }
  t->check_rec = alloc_n<unsigned long long>(a, 4);
  GB_CK(cudaMemsetAsync(t->check_rec, 0, 4 * sizeof(unsigned long long), s));
  mark(FMM_PH_BUILD_OPS, 1);
  mark(FMM_PH_BUILD_TOTAL, 1);
  long long nitem[2] = {0, 0}, tail[4] = {0, 0, 0, 0};
  if (t->p2p_nitem) GB_CK(cudaMemcpyAsync(nitem, t->p2p_nitem, sizeof(nitem), cudaMemcpyDeviceToHost, s));
  GB_CK(cudaMemcpyAsync(tail, t->d_tail, sizeof(tail), cudaMemcpyDeviceToHost, s));
  check_scan_error(a, s);  // synchronises
  t->p2p_nitem_host = nitem[0];
  t->p2p_nbig_host = nitem[1];
  t->n_p2p_ranges = tail[0];
  t->p2p_body_pairs = tail[1] - t->N;
  if (tail[2]) fail(FMM_ERR_RANGE, "translation operator overflows the working precision");
  if (t->m2l_engine == 1) finish_m2l_chunks(t, tail[3]);
  t->lim = Lim{t->N, t->ncell, t->nleaf, t->Kp, t->ntile, t->nentry, t->nclass, t->n_p2p_ranges, t->check_rec};
  t->build_syncs = a.nsync;
  if (timing)
    for (int ph : {FMM_PH_BUILD_TOTAL, FMM_PH_BUILD_TREE, FMM_PH_BUILD_LISTS, FMM_PH_BUILD_PLAN, FMM_PH_BUILD_OPS})
      cudaEventElapsedTime(&t->ms[ph], t->ev[2 * ph], t->ev[2 * ph + 1]);
}

constexpr uint32_t kKnownFlags = FMM_FLAG_CIRCUMSCRIBED | FMM_FLAG_TIMING | FMM_FLAG_M2L_CUDA_CORE |
                                 FMM_FLAG_SORTED_PLAN | FMM_FLAG_SERIAL_PHASES | FMM_FLAG_MUTUAL_P2P |
                                 FMM_FLAG_TIGHT_MAC | FMM_FLAG_FITTED_CENTRES;

template <class R>
int build_common(const R* xyzq, int64_t n, int p, double theta, int ncrit, uint32_t flags,
                 const fmm_allocator* alloc, fmm_stream stream, fmm_tree** out) {
  if (out) *out = nullptr;
  if (!xyzq || !out || n < 1 || n > 0x7fffffffll || p < 1 || p > kMaxP || !(theta > 0.0) ||
      !(theta < 1.0) || ncrit < 1 || (flags & ~kKnownFlags))
    return FMM_ERR_ARG;
  if (alloc && (!alloc->alloc || !alloc->free)) return FMM_ERR_ARG;
  fmm_tree* t = new (std::nothrow) fmm_tree();
  if (!t) return FMM_ERR_OOM;
  t->N = n;
  t->p = p;
  t->theta = theta;
  t->ncrit = ncrit;
  t->flags = flags;
  t->stream = (cudaStream_t)stream;
  t->arena.stream = t->stream;
  if (alloc) {
    t->arena.user = *alloc;
    t->arena.has_user = true;
  }
  try {
    create_tree<R>(t, xyzq);
  } catch (const Error& e) {
    release_tree(t);
    return to_code(e);
  } catch (const std::bad_alloc&) {
    release_tree(t);
    return FMM_ERR_OOM;
  }
  *out = t;
  return FMM_OK;
}

struct PhaseTimer {
  fmm_tree* t;
  cudaStream_t s;
  bool on;
  void begin(int ph) {
    if (on) cudaEventRecord(t->ev[2 * ph], s);
  }
  void end(int ph) {
    if (on) cudaEventRecord(t->ev[2 * ph + 1], s);
  }
};

// One FMM pass with the charges currently in t->work.
template <class R>
void run_pass(fmm_tree* t, cudaStream_t s, int mode, R* a, R* b) {
  const bool timing = (t->flags & FMM_FLAG_TIMING) != 0;
  const bool serial = (t->flags & FMM_FLAG_SERIAL_PHASES) != 0;
  // Concurrent mode: the far field runs on the library's highest-priority
  // stream and the near field on its lowest-priority stream, both forked
  // from the caller's stream and joined back before L2P.  P2P fills the GPU
  // during P2M and M2M; once M2L is launched its CTAs (one per SM, most of
  // its shared memory) are dispatched first as P2P blocks retire, and P2P
  // blocks fill the registers, shared memory and issue slots they leave
  // free.  Serial mode runs every phase on the caller's stream, P2P first.
  cudaStream_t fs = serial ? s : t->far;
  cudaStream_t ps = serial ? s : t->side;
  PhaseTimer Ttot{t, s, timing}, T{t, fs, timing}, Tp{t, ps, timing};
  Ttot.begin(FMM_PH_EVAL_TOTAL);
  auto near_field = [&] {
    if (!serial) GB_CK(cudaStreamWaitEvent(ps, t->fork, 0));
    Tp.begin(FMM_PH_P2P);
    launch_p2p<R>(t, ps);
    Tp.end(FMM_PH_P2P);
    if (!serial) GB_CK(cudaEventRecord(t->join, ps));
  };
  if (!serial) {
    GB_CK(cudaEventRecord(t->fork, s));
    GB_CK(cudaStreamWaitEvent(fs, t->fork, 0));
  }
  near_field();
  // far field
  GB_CK(cudaMemsetAsync(t->L, 0, sizeof(R) * (size_t)t->ncell * t->Kp, fs));
  T.begin(FMM_PH_P2M);
  launch_p2m<R>(t, fs);
  T.end(FMM_PH_P2M);
  const bool fitted = t->m2l_engine == 3;
  T.begin(FMM_PH_M2M);
  for (int l = t->nlevel - 2; l >= 0; --l) {
    if (fitted) launch_m2m_fit<R>(t, l, fs);
    else launch_m2m<R>(t, l, fs);
  }
  T.end(FMM_PH_M2M);
  T.begin(FMM_PH_M2L);
  if (fitted) {
    launch_m2l_fit<R>(t, fs);
  } else if (t->m2l_engine == 1) {
    launch_split_tf32(t, fs);
    launch_m2l_tcgen05(t, fs);
  } else {
    launch_m2l_cuda_core<R>(t, fs);
  }
  T.end(FMM_PH_M2L);
  T.begin(FMM_PH_L2L);
  for (int l = 1; l < t->nlevel; ++l) {
    if (fitted) launch_l2l_fit<R>(t, l, fs);
    else launch_l2l<R>(t, l, fs);
  }
  T.end(FMM_PH_L2L);
  if (!serial) {
    GB_CK(cudaEventRecord(t->join_far, fs));
    GB_CK(cudaStreamWaitEvent(s, t->join_far, 0));
    GB_CK(cudaStreamWaitEvent(s, t->join, 0));
  }
  Ttot.begin(FMM_PH_L2P);
  launch_l2p_finalize<R>(t, mode, a, b, s);
  Ttot.end(FMM_PH_L2P);
  Ttot.end(FMM_PH_EVAL_TOTAL);
}

template <class R>
int evaluate_common(fmm_tree* t, const R* q, R* pot, R* force, fmm_stream stream) {
  if (!t || !pot) return FMM_ERR_ARG;
  if (t->precision != (int)(8 * sizeof(R))) return FMM_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    if (q) launch_set_charges<R>(t, q, s);
    else GB_CK(cudaMemcpyAsync(t->work, t->bodies, sizeof(R) * 4 * (size_t)t->N, cudaMemcpyDeviceToDevice, s));
    run_pass<R>(t, s, 0, pot, force);
    GB_CK(cudaEventRecord(t->pass_done, s));
    t->evaluations++;
  } catch (const Error& e) {
    return to_code(e);
  }
  return FMM_OK;
}

template <class R>
int backward_common(fmm_tree* t, const R* w, R* dq, R* dx, fmm_stream stream) {
  if (!t || !w || !dq || !dx) return FMM_ERR_ARG;
  if (t->precision != (int)(8 * sizeof(R))) return FMM_ERR_STATE;
  if (t->evaluations == 0) return FMM_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  try {
    launch_set_charges<R>(t, w, s);
    run_pass<R>(t, s, 1, dq, dx);
    GB_CK(cudaEventRecord(t->pass_done, s));
  } catch (const Error& e) {
    return to_code(e);
  }
  return FMM_OK;
}

// host: waits for the tree's last evaluate / backward and reads its device
// error word; -1 if the wait or the copy failed
int read_device_errors(const fmm_tree* t) {
  if (!t->dev_err) return 0;
  if (t->pass_done && cudaEventSynchronize(t->pass_done) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  int h = 0;
  if (cudaMemcpy(&h, t->dev_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return h;
}

}  // namespace

extern "C" {

int fmm_build(const float* xyzq, int64_t n, int p, double theta, int ncrit, uint32_t flags,
              const fmm_allocator* alloc, fmm_stream stream, fmm_tree** out) {
  return build_common<float>(xyzq, n, p, theta, ncrit, flags, alloc, stream, out);
}

int fmm_build_f64(const double* xyzq, int64_t n, int p, double theta, int ncrit, uint32_t flags,
                  const fmm_allocator* alloc, fmm_stream stream, fmm_tree** out) {
  return build_common<double>(xyzq, n, p, theta, ncrit, flags, alloc, stream, out);
}

int fmm_evaluate(fmm_tree* t, const float* q, float* pot, float* force, fmm_stream stream) {
  return evaluate_common<float>(t, q, pot, force, stream);
}

int fmm_evaluate_f64(fmm_tree* t, const double* q, double* pot, double* force, fmm_stream stream) {
  return evaluate_common<double>(t, q, pot, force, stream);
}

int fmm_backward(fmm_tree* t, const float* w, float* dq, float* dx, fmm_stream stream) {
  return backward_common<float>(t, w, dq, dx, stream);
}

int fmm_backward_f64(fmm_tree* t, const double* w, double* dq, double* dx, fmm_stream stream) {
  return backward_common<double>(t, w, dq, dx, stream);
}

int fmm_solve_host(const float* xyzq_h, const float* w_h, int64_t n, int p, double theta, int ncrit,
                   uint32_t flags, float* pot_h, float* force_h, float* dq_h, float* dx_h,
                   fmm_stream stream) {
  if (!xyzq_h || !pot_h || n < 1 || n > 0x7fffffffll) return FMM_ERR_ARG;
  if (w_h && (!dq_h || !dx_h)) return FMM_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  float *d_x = nullptr, *d_w = nullptr, *d_pot = nullptr, *d_force = nullptr, *d_dq = nullptr, *d_dx = nullptr;
  fmm_tree* t = nullptr;
  int rc = FMM_OK;
  cudaMemPool_t pool = nullptr;
  try {
    pool = library_pool();
  } catch (const Error& e) {
    return to_code(e);
  }
  auto mal = [&](float** p, size_t count) {
    if (rc != FMM_OK) return;
    if (cudaMallocFromPoolAsync((void**)p, sizeof(float) * count, pool, s) != cudaSuccess) {
      cudaGetLastError();
      rc = FMM_ERR_OOM;
    }
  };
  mal(&d_x, 4 * (size_t)n);
  mal(&d_pot, (size_t)n);
  if (force_h) mal(&d_force, 3 * (size_t)n);
  if (w_h) {
    mal(&d_w, (size_t)n);
    mal(&d_dq, (size_t)n);
    mal(&d_dx, 3 * (size_t)n);
  }
  if (rc == FMM_OK && cudaMemcpyAsync(d_x, xyzq_h, sizeof(float) * 4 * n, cudaMemcpyHostToDevice, s) != cudaSuccess)
    rc = FMM_ERR_CUDA;
  if (rc == FMM_OK && w_h && cudaMemcpyAsync(d_w, w_h, sizeof(float) * n, cudaMemcpyHostToDevice, s) != cudaSuccess)
    rc = FMM_ERR_CUDA;
  if (rc == FMM_OK) rc = fmm_build(d_x, n, p, theta, ncrit, flags, nullptr, stream, &t);
  if (rc == FMM_OK) rc = fmm_evaluate(t, nullptr, d_pot, d_force, stream);
  if (rc == FMM_OK && w_h) rc = fmm_backward(t, d_w, d_dq, d_dx, stream);
  if (rc == FMM_OK) rc = fmm_check(t);
  auto back = [&](float* h, const float* d, size_t count) {
    if (rc == FMM_OK && h && cudaMemcpyAsync(h, d, sizeof(float) * count, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      rc = FMM_ERR_CUDA;
  };
  back(pot_h, d_pot, (size_t)n);
  if (force_h) back(force_h, d_force, 3 * (size_t)n);
  if (w_h) {
    back(dq_h, d_dq, (size_t)n);
    back(dx_h, d_dx, 3 * (size_t)n);
  }
  if (t) fmm_destroy(t);
  float* all[6] = {d_x, d_w, d_pot, d_force, d_dq, d_dx};
  for (float* p : all)
    if (p) cudaFreeAsync(p, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && rc == FMM_OK) rc = FMM_ERR_CUDA;
  cudaGetLastError();
  return rc;
}

int fmm_get_stats(const fmm_tree* tc, fmm_stats* o) {
  if (!tc || !o) return FMM_ERR_ARG;
  fmm_tree* t = const_cast<fmm_tree*>(tc);
  std::memset(o, 0, sizeof(*o));
  o->n_bodies = t->N;
  o->n_cells = t->ncell;
  o->n_leaves = t->nleaf;
  o->n_levels = t->nlevel;
  o->n_p2p = t->n_p2p;
  o->n_p2p_ranges = t->n_p2p_ranges;
  o->n_p2p_body_pairs = t->p2p_body_pairs;
  o->n_m2l = t->n_m2l;
  o->n_m2l_classes = t->nclass;
  o->n_m2l_tiles = t->ntile;
  o->n_m2l_slots = t->nentry * kTile;
  o->p = t->p;
  o->K = t->K;
  o->ncrit = t->ncrit;
  o->precision_bits = t->precision;
  o->theta = t->theta;
  o->flags = t->flags;
  o->m2l_engine = t->m2l_engine == 1 && t->m2l_quad ? 2 : t->m2l_engine;
  o->workspace_bytes = (int64_t)t->arena.bytes;
  o->evaluations = t->evaluations;
  const int derr = read_device_errors(t);
  if (derr < 0) return FMM_ERR_CUDA;
  o->device_errors = derr;
  o->build_host_syncs = t->build_syncs;
  if ((t->flags & FMM_FLAG_TIMING) && t->evaluations > 0) {
    if (cudaEventSynchronize(t->ev[2 * FMM_PH_EVAL_TOTAL + 1]) != cudaSuccess) {
      cudaGetLastError();
      return FMM_ERR_CUDA;
    }

    for (int ph = 0; ph < FMM_PH_BUILD_TOTAL; ++ph) {  // evaluate phases; build times are set by fmm_build
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, t->ev[2 * ph], t->ev[2 * ph + 1]) == cudaSuccess) t->ms[ph] = ms;
      else cudaGetLastError();
    }
  }
  for (int ph = 0; ph < FMM_PH_COUNT; ++ph) o->ms[ph] = t->ms[ph];
  return derr ? FMM_ERR_TIMEOUT : FMM_OK;
}

int fmm_check(const fmm_tree* t) {
  if (!t) return FMM_ERR_ARG;
  const int derr = read_device_errors(t);
  if (derr < 0) return FMM_ERR_CUDA;
  return derr ? FMM_ERR_TIMEOUT : FMM_OK;
}


int fmm_destroy(fmm_tree* t) {
  if (!t) return FMM_OK;
  // the caller's streams of earlier calls: wait for all of the device's work
  // on this tree's buffers before they are released
  cudaError_t e = cudaDeviceSynchronize();
  release_tree(t);
  return e == cudaSuccess ? FMM_OK : FMM_ERR_CUDA;
}

const char* fmm_strerror(int code) {
  switch (code) {
    case FMM_OK: return "ok";
    case FMM_ERR_ARG: return "invalid argument";
    case FMM_ERR_NONFINITE: return "non-finite position or charge";
    case FMM_ERR_OOM: return "out of device memory";
    case FMM_ERR_CUDA: return "CUDA error";
    case FMM_ERR_TIMEOUT: return "bounded device wait timed out";
    case FMM_ERR_STATE: return "call out of order or wrong precision";
    case FMM_ERR_RANGE: return "operator not representable in the working precision";
    default: return "unknown error";
  }
}

int fmm_get_root(const fmm_tree* t, double* out) {
  if (!t || !out) return FMM_ERR_ARG;
  for (int k = 0; k < 3; ++k) {
    out[k] = t->root.lo[k];
    out[3 + k] = t->root.hi[k];
    out[6 + k] = t->root.centre[k];
    out[10 + k] = t->root.corner[k];
  }
  out[9] = t->root.H;
  return FMM_OK;
}

int fmm_get_keys(const fmm_tree* t, uint64_t* keys, int32_t* perm, fmm_stream stream) {
  if (!t || !keys || !perm) return FMM_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(keys, t->keys, sizeof(uint64_t) * t->N, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(perm, t->perm, sizeof(int32_t) * t->N, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
    cudaGetLastError();
    return FMM_ERR_CUDA;
  }
  return FMM_OK;
}

int fmm_get_cells(const fmm_tree* t, int32_t* cells, fmm_stream stream) {
  if (!t || !cells) return FMM_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int32_t* rows[9] = {t->c.level, t->c.ix, t->c.iy, t->c.iz, t->c.bbeg, t->c.bend, t->c.cbeg, t->c.nch, t->c.parent};
  for (int r = 0; r < 9; ++r)
    if (cudaMemcpyAsync(cells + (int64_t)r * t->ncell, rows[r], sizeof(int32_t) * t->ncell,
                        cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
      cudaGetLastError();
      return FMM_ERR_CUDA;
    }
  return FMM_OK;
}

int fmm_get_lists(const fmm_tree* tc, int32_t* p2p_tgt, int32_t* p2p_src, int32_t* m2l_tgt, int32_t* m2l_src,
                  fmm_stream stream) {
  if (!tc || !p2p_tgt || !p2p_src || (tc->n_m2l && (!m2l_tgt || !m2l_src))) return FMM_ERR_ARG;
  fmm_tree* t = const_cast<fmm_tree*>(tc);
  cudaStream_t s = (cudaStream_t)stream;
  // the tree keeps traversal order; sort copies by (target, source) on the
  // caller's stream (workspace from the tree's allocator)
  cudaStream_t keep = t->arena.stream;
  t->arena.stream = s;
  int rc = FMM_OK;
  try {
    sort_pairs_copy(t->arena, t->p2p_tgt, t->p2p_src, t->n_p2p, t->ncell, p2p_tgt, p2p_src, s);
    sort_pairs_copy(t->arena, t->m2l_tgt, t->m2l_src, t->n_m2l, t->ncell, m2l_tgt, m2l_src, s);
  } catch (const Error& e) {
    rc = e.code;
  }
  t->arena.stream = keep;
  return rc;
}

int fmm_get_expansions(const fmm_tree* t, void* M, void* L, fmm_stream stream) {
  if (!t) return FMM_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t rs = t->precision == 64 ? 8 : 4;
  // rows are stored with a padded stride Kp; copy out K per row
  if (M && cudaMemcpy2DAsync(M, rs * t->K, t->M, rs * t->Kp, rs * t->K, t->ncell, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
    cudaGetLastError();
    return FMM_ERR_CUDA;
  }
  if (L && cudaMemcpy2DAsync(L, rs * t->K, t->L, rs * t->Kp, rs * t->K, t->ncell, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
    cudaGetLastError();
    return FMM_ERR_CUDA;
  }
  return FMM_OK;
}

int fmm_debug_checks(const fmm_tree* t, int64_t* out) {
  if (!t || !out) return FMM_ERR_ARG;
  unsigned long long h[4] = {0, 0, 0, 0};
  if (cudaMemcpy(h, t->check_rec, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return FMM_ERR_CUDA;
  }
  for (int k = 0; k < 4; ++k) out[k] = (int64_t)h[k];
#ifdef GBFMM_CHECKED
  return 1;
#else
  return FMM_OK;
#endif
}

int fmm_get_plan(const fmm_tree* t, int32_t* tile_tgt, int32_t* tile_eptr, int32_t* entry_class,
                 int32_t* entry_src, int32_t* p2p_rptr, int32_t* p2p_ranges, fmm_stream stream) {
  if (!t) return FMM_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  struct Cp {
    void* dst;
    const void* src;
    size_t bytes;
  } cps[6] = {
      {tile_tgt, t->tile_tgt, sizeof(int32_t) * (size_t)t->ntile * kTile},
      {tile_eptr, t->tile_eptr, sizeof(int32_t) * (size_t)(t->ntile + 1)},
      {entry_class, t->entry_class, sizeof(int32_t) * (size_t)t->nentry},
      {entry_src, t->entry_src, sizeof(int32_t) * (size_t)t->nentry * kTile},
      {p2p_rptr, t->p2p_rptr, sizeof(int32_t) * (size_t)(t->nleaf + 1)},
      {p2p_ranges, t->p2p_ranges, sizeof(int2) * (size_t)t->n_p2p_ranges},
  };
  for (auto& c : cps) {
    if (!c.dst || !c.src || c.bytes == 0) continue;
    if (cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
      cudaGetLastError();
      return FMM_ERR_CUDA;
    }
  }
  return FMM_OK;
}

}  // extern "C"
