"""ctypes binding of libgbfmm.so (argument marshalling only).

Every step of the FMM runs in the library's CUDA kernels; this module only
passes device pointers of torch tensors, the current torch stream and sizes
through the C ABI declared in ``include/gbfmm.h``.  The library is loaded on
first use; if it is missing this raises (there is no fallback).
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgbfmm_checked.so" if os.environ.get("GBFMM_CHECKED") == "1"
                        else ("libgbfmm_traced.so" if os.environ.get("GBFMM_TRACE") == "1" else "libgbfmm.so"))
_lib = None

FMM_FLAG_CIRCUMSCRIBED = 1
FMM_FLAG_TIMING = 2
FMM_FLAG_M2L_CUDA_CORE = 4
FMM_FLAG_SORTED_PLAN = 8
FMM_FLAG_SERIAL_PHASES = 16
FMM_FLAG_MUTUAL_P2P = 32
FMM_FLAG_TIGHT_MAC = 64
FMM_FLAG_FITTED_CENTRES = 128

PHASES = ("p2m", "m2m", "m2l", "l2l", "p2p", "l2p", "eval_total", "build_total",
          "build_tree", "build_lists", "build_plan", "build_ops")

_ERRORS = {0: "ok", -1: "FMM_ERR_ARG", -2: "FMM_ERR_NONFINITE", -3: "FMM_ERR_OOM", -4: "FMM_ERR_CUDA",
           -5: "FMM_ERR_TIMEOUT", -6: "FMM_ERR_STATE", -7: "FMM_ERR_RANGE"}


class FMMError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        self.name = _ERRORS.get(code, str(code))
        detail = lib().fmm_last_error().decode(errors="replace")
        super().__init__(f"{where}: {self.name} ({lib().fmm_strerror(code).decode()}) {detail}")


class Stats(ctypes.Structure):
    _fields_ = [("n_bodies", ctypes.c_int64), ("n_cells", ctypes.c_int64), ("n_leaves", ctypes.c_int64),
                ("n_levels", ctypes.c_int64), ("n_p2p", ctypes.c_int64), ("n_p2p_ranges", ctypes.c_int64),
                ("n_p2p_body_pairs", ctypes.c_int64), ("n_m2l", ctypes.c_int64),
                ("n_m2l_classes", ctypes.c_int64), ("n_m2l_tiles", ctypes.c_int64),
                ("n_m2l_slots", ctypes.c_int64), ("p", ctypes.c_int32), ("K", ctypes.c_int32),
                ("ncrit", ctypes.c_int32), ("precision_bits", ctypes.c_int32), ("theta", ctypes.c_double),
                ("flags", ctypes.c_uint32), ("m2l_engine", ctypes.c_int32),
                ("workspace_bytes", ctypes.c_int64), ("evaluations", ctypes.c_int32),
                ("device_errors", ctypes.c_int32), ("build_host_syncs", ctypes.c_int32),
                ("ms", ctypes.c_float * len(PHASES))]


_V = ctypes.c_void_p
_I64 = ctypes.c_int64

# fmm_allocator: stream-ordered alloc / free callbacks and their context
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    """The C ABI's fmm_allocator.  Keep the callback objects alive for as long
    as a tree built with it exists."""
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


def lib():
    """Load libgbfmm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "fmm_build": [_V, _I64, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_uint32, _V, _V,
                          ctypes.POINTER(_V)],
            "fmm_build_f64": [_V, _I64, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_uint32, _V, _V,
                              ctypes.POINTER(_V)],
            "fmm_evaluate": [_V, _V, _V, _V, _V],
            "fmm_evaluate_f64": [_V, _V, _V, _V, _V],
            "fmm_backward": [_V, _V, _V, _V, _V],
            "fmm_backward_f64": [_V, _V, _V, _V, _V],
            "fmm_solve_host": [_V, _V, _I64, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_uint32, _V,
                               _V, _V, _V, _V],
            "fmm_get_stats": [_V, ctypes.POINTER(Stats)],
            "fmm_destroy": [_V],
            "fmm_get_root": [_V, _V],
            "fmm_get_keys": [_V, _V, _V, _V],
            "fmm_get_cells": [_V, _V, _V],
            "fmm_get_lists": [_V, _V, _V, _V, _V, _V],
            "fmm_get_expansions": [_V, _V, _V, _V],
            "fmm_direct_f64": [_V, _I64, _V, _I64, _V, _V, _V],
            "fmm_get_plan": [_V, _V, _V, _V, _V, _V, _V, _V],
            "fmm_debug_checks": [_V, _V],
            "fmm_check": [_V],
            "fmm_debug_m2l_trace": [_V],
            "fmm_debug_scan_fault": [ctypes.c_int],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.fmm_launch_count.argtypes = []
        L.fmm_launch_count.restype = ctypes.c_int64
        L.fmm_last_error.argtypes = []
        L.fmm_last_error.restype = ctypes.c_char_p
        L.fmm_strerror.argtypes = [ctypes.c_int]
        L.fmm_strerror.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(rc: int, where: str):
    if rc != 0:
        raise FMMError(rc, where)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _dev_tensor(t: torch.Tensor, dtype, shape, what):
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError(f"{what} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{what} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t.contiguous()


class Tree:
    """An FMM tree built on the GPU (fmm_build / fmm_build_f64).

    xyzq: CUDA tensor (N, 4) of x, y, z, q; float32 selects the single
    precision path, float64 the double precision one.
    """

    def __init__(self, xyzq: torch.Tensor, p: int, theta: float, ncrit: int, flags: int = 0,
                 allocator: Optional[Allocator] = None):
        L = lib()
        if not (isinstance(xyzq, torch.Tensor) and xyzq.is_cuda and xyzq.dim() == 2 and xyzq.shape[1] == 4):
            raise ValueError("xyzq must be a CUDA tensor of shape (N, 4)")
        if xyzq.dtype not in (torch.float32, torch.float64):
            raise TypeError("xyzq must be float32 or float64")
        self.dtype = xyzq.dtype
        self.device = xyzq.device
        self.N = xyzq.shape[0]
        self.p = int(p)
        x = xyzq.contiguous()
        h = ctypes.c_void_p()
        build = L.fmm_build if self.dtype == torch.float32 else L.fmm_build_f64
        with torch.cuda.device(self.device):
            rc = build(_ptr(x), self.N, self.p, float(theta), int(ncrit), int(flags),
                       None if allocator is None else ctypes.byref(allocator), _stream(self.device),
                       ctypes.byref(h))
        _check(rc, "fmm_build")
        self._h = h
        self._allocator = allocator  # the callbacks must outlive the tree

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().fmm_destroy(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def evaluate(self, q: Optional[torch.Tensor] = None, force: bool = True):
        """(pot (N,), force (N, 3) or None); force = -grad phi."""
        L = lib()
        qq = None if q is None else _dev_tensor(q, self.dtype, (self.N,), "q")
        pot = torch.empty(self.N, dtype=self.dtype, device=self.device)
        f = torch.empty((self.N, 3), dtype=self.dtype, device=self.device) if force else None
        fn = L.fmm_evaluate if self.dtype == torch.float32 else L.fmm_evaluate_f64
        with torch.cuda.device(self.device):
            _check(fn(self._h, _ptr(qq), _ptr(pot), _ptr(f), _stream(self.device)), "fmm_evaluate")
        return pot, f

    def backward(self, w: torch.Tensor):
        """Adjoint of L with dL/dphi = w: (dL/dq (N,), dL/dx (N, 3))."""
        L = lib()
        ww = _dev_tensor(w, self.dtype, (self.N,), "w")
        dq = torch.empty(self.N, dtype=self.dtype, device=self.device)
        dx = torch.empty((self.N, 3), dtype=self.dtype, device=self.device)
        fn = L.fmm_backward if self.dtype == torch.float32 else L.fmm_backward_f64
        with torch.cuda.device(self.device):
            _check(fn(self._h, _ptr(ww), _ptr(dq), _ptr(dx), _stream(self.device)), "fmm_backward")
        return dq, dx

    def check(self):
        """Raises FMMError (FMM_ERR_TIMEOUT) if a bounded device wait of any
        pass on this tree gave up (fmm_check); waits for the last pass."""
        _check(lib().fmm_check(self._h), "fmm_check")

    def stats(self) -> dict:
        s = Stats()
        _check(lib().fmm_get_stats(self._h, ctypes.byref(s)), "fmm_get_stats")
        out = {k: getattr(s, k) for k, _ in Stats._fields_ if k != "ms"}
        out["ms"] = {PHASES[i]: float(s.ms[i]) for i in range(len(PHASES))}
        return out

    # ---- inspection
    def root(self) -> dict:
        out = np.zeros(13)
        _check(lib().fmm_get_root(self._h, out.ctypes.data_as(ctypes.c_void_p)), "fmm_get_root")
        return {"lo": out[0:3], "hi": out[3:6], "centre": out[6:9], "H": out[9], "corner": out[10:13]}

    def keys(self):
        k = torch.empty(self.N, dtype=torch.int64, device=self.device)
        perm = torch.empty(self.N, dtype=torch.int32, device=self.device)
        with torch.cuda.device(self.device):
            _check(lib().fmm_get_keys(self._h, _ptr(k), _ptr(perm), _stream(self.device)), "fmm_get_keys")
        return k.cpu().numpy().view(np.uint64), perm.cpu().numpy()

    def cells(self) -> dict:
        n = self.stats()["n_cells"]
        c = torch.empty((9, n), dtype=torch.int32, device=self.device)
        with torch.cuda.device(self.device):
            _check(lib().fmm_get_cells(self._h, _ptr(c), _stream(self.device)), "fmm_get_cells")
        c = c.cpu().numpy()
        names = ("level", "ix", "iy", "iz", "body_begin", "body_end", "child_begin", "child_count", "parent")
        return {k: c[i] for i, k in enumerate(names)}

    def lists(self) -> dict:
        st = self.stats()
        a = [torch.empty(st["n_p2p"], dtype=torch.int32, device=self.device) for _ in range(2)]
        b = [torch.empty(max(1, st["n_m2l"]), dtype=torch.int32, device=self.device) for _ in range(2)]
        with torch.cuda.device(self.device):
            _check(lib().fmm_get_lists(self._h, *(_ptr(x) for x in a + b), _stream(self.device)), "fmm_get_lists")
        n = st["n_m2l"]
        return {"p2p_tgt": a[0].cpu().numpy(), "p2p_src": a[1].cpu().numpy(),
                "m2l_tgt": b[0].cpu().numpy()[:n], "m2l_src": b[1].cpu().numpy()[:n]}

    def debug_checks(self) -> dict:
        """Self-check record (checked build only): first bad access, count."""
        out = np.zeros(4, np.int64)
        checked = lib().fmm_debug_checks(self._h, out.ctypes.data_as(ctypes.c_void_p))
        return {"checked": checked == 1, "site": int(out[0]), "index": int(out[1]), "bound": int(out[2]),
                "count": int(out[3])}

    def plan(self) -> dict:
        """M2L tiles/entries and P2P source ranges (host numpy arrays)."""
        st = self.stats()
        nt, ne = st["n_m2l_tiles"], st["n_m2l_slots"] // 128
        z = lambda n: torch.empty(max(1, n), dtype=torch.int32, device=self.device)
        a = {"tile_tgt": z(nt * 128), "tile_eptr": z(nt + 1), "entry_class": z(ne), "entry_src": z(ne * 128),
             "p2p_rptr": z(st["n_leaves"] + 1), "p2p_ranges": z(2 * st["n_p2p_ranges"])}
        with torch.cuda.device(self.device):
            _check(lib().fmm_get_plan(self._h, *(_ptr(a[k]) for k in ("tile_tgt", "tile_eptr", "entry_class",
                                                                       "entry_src", "p2p_rptr", "p2p_ranges")),
                                      _stream(self.device)), "fmm_get_plan")
        n = {"tile_tgt": nt * 128, "tile_eptr": nt + 1, "entry_class": ne, "entry_src": ne * 128,
             "p2p_rptr": st["n_leaves"] + 1, "p2p_ranges": 2 * st["n_p2p_ranges"]}
        out = {k: v.cpu().numpy()[:n[k]] for k, v in a.items()}
        out["p2p_ranges"] = out["p2p_ranges"].reshape(-1, 2)
        out["entry_src"] = out["entry_src"].reshape(-1, 128)
        out["tile_tgt"] = out["tile_tgt"].reshape(-1, 128)
        return out

    def expansions(self):
        """(M, L) real-packed and scaled, shape (n_cells, p*p)."""
        st = self.stats()
        M = torch.empty((st["n_cells"], st["K"]), dtype=self.dtype, device=self.device)
        Lx = torch.empty_like(M)
        with torch.cuda.device(self.device):
            _check(lib().fmm_get_expansions(self._h, _ptr(M), _ptr(Lx), _stream(self.device)),
                   "fmm_get_expansions")
        return M.cpu().numpy(), Lx.cpu().numpy()


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(lib().fmm_launch_count())


def direct_f64(xyzq: torch.Tensor, targets: torch.Tensor, force: bool = True):
    """Double-precision direct sum at the target input indices
    (fmm_direct_f64): (pot (nt,), force (nt, 3)) as float64 CUDA tensors."""
    x = _dev_tensor(xyzq, torch.float32, (xyzq.shape[0], 4), "xyzq")
    if targets.dim() != 1:
        raise ValueError("targets must be one-dimensional")
    tg = targets.to(device=x.device, dtype=torch.int32).contiguous()
    nt = tg.shape[0]
    pot = torch.empty(nt, dtype=torch.float64, device=x.device)
    f = torch.empty((nt, 3), dtype=torch.float64, device=x.device) if force else None
    with torch.cuda.device(x.device):
        _check(lib().fmm_direct_f64(_ptr(x), x.shape[0], _ptr(tg), nt, _ptr(pot), _ptr(f), _stream(x.device)),
               "fmm_direct_f64")
    return pot, f


def solve_host(xyzq: np.ndarray, w: Optional[np.ndarray], p: int, theta: float, ncrit: int,
               flags: int = 0, force: bool = True, stream: Optional[torch.cuda.Stream] = None) -> dict:
    """One whole step through host buffers (fmm_solve_host): build, evaluate
    and, when w is given, the backward pass, copies included."""
    x = np.ascontiguousarray(xyzq, dtype=np.float32)
    if x.ndim != 2 or x.shape[1] != 4 or x.shape[0] < 1:
        raise ValueError(f"xyzq must have shape (N, 4) with N >= 1, got {x.shape}")
    N = x.shape[0]
    if w is not None and np.shape(w) != (N,):
        raise ValueError(f"w must have shape ({N},), got {np.shape(w)}")
    pot = np.empty(N, np.float32)
    frc = np.empty((N, 3), np.float32) if force else None
    ww = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
    dq = np.empty(N, np.float32) if ww is not None else None
    dx = np.empty((N, 3), np.float32) if ww is not None else None
    vp = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)
    s = ctypes.c_void_p(stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream)
    _check(lib().fmm_solve_host(vp(x), vp(ww), N, int(p), float(theta), int(ncrit), int(flags), vp(pot),
                                vp(frc), vp(dq), vp(dx), s), "fmm_solve_host")
    return {"pot": pot, "force": frc, "dq": dq, "dx": dx}


class _FMMFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, q, p, theta, ncrit):
        xyzq = torch.cat([x.detach(), q.detach()[:, None]], dim=1).contiguous()
        tree = Tree(xyzq, p, theta, ncrit)
        pot, force = tree.evaluate()
        ctx.tree = tree
        ctx.mark_non_differentiable(force)
        return pot, force

    @staticmethod
    def backward(ctx, gpot, gforce):
        if gforce is not None and bool((gforce != 0).any()):
            raise NotImplementedError("gradients flow from the potential only")
        if gpot is None:
            return None, None, None, None, None
        dq, dx = ctx.tree.backward(gpot.contiguous())
        return dx, dq, None, None, None


class FMM:
    """Differentiable FMM: ``FMM(p, theta, ncrit)(x, q) -> (phi, force)``.

    x: (N, 3) and q: (N,) CUDA tensors (float32 or float64).  Gradients of a
    loss of ``phi`` reach x and q through the hand-written adjoint
    (fmm_backward) on the frozen tree.
    """

    def __init__(self, p: int, theta: float, ncrit: int):
        self.p, self.theta, self.ncrit = int(p), float(theta), int(ncrit)

    def __call__(self, x: torch.Tensor, q: torch.Tensor):
        return _FMMFunction.apply(x, q, self.p, self.theta, self.ncrit)
