"""Double-precision CPU oracle of the FMM hot path (test infrastructure).

Only the tests, the package smoke check and the CPU-baseline leg of the
benchmark may import this module.  The product (the CUDA library and its
Python binding) never imports, links or runs anything here, and this module
imports nothing from the product.  It wraps ``fmm_oracle.cpp`` through
ctypes; :func:`build` compiles it with the host C++ compiler.

Everything here is plain double precision.  Inputs are widened exactly from
whatever the caller passes (the workloads are float32).  Outputs are the
potential ``phi`` and its gradient ``grad`` (the force per unit charge is
``-grad``), with the conventions stated at the top of ``fmm_oracle.cpp``.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmm_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_I32 = ctypes.POINTER(ctypes.c_int32)
_U64 = ctypes.POINTER(ctypes.c_uint64)


def compile_library(src: str, out: str) -> None:
    """Compile an oracle source file into a shared library (g++, OpenMP, no FMA
    contraction: the tree build's floating-point steps must round as written)."""
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fPIC",
           "-shared", "-o", out, src]
    subprocess.run(cmd, check=True)


def build(force: bool = False) -> str:
    """Compile the oracle shared library next to its source when it is stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        compile_library(_SRC, tmp)
        os.replace(tmp, _LIB)
    return _LIB


def use_library(path: str) -> None:
    """Make this module call another build of the oracle's source.  The
    mutation tests plant one mistake in a copy of ``fmm_oracle.cpp``, build it
    with :func:`compile_library` and run the pins against it through here."""
    global _lib
    _lib = _load(path)


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = _load(_LIB)
    return _lib


def _load(path: str):
    L = ctypes.CDLL(path)
    L.orc_set_threads.argtypes = [ctypes.c_int]
    L.orc_build.argtypes = [_D, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                            ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
    L.orc_set_order.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.orc_centres.argtypes = [ctypes.c_void_p, _D]
    L.orc_free.argtypes = [ctypes.c_void_p]
    L.orc_free.restype = None
    L.orc_info.argtypes = [ctypes.c_void_p, _I64]
    L.orc_root.argtypes = [ctypes.c_void_p, _D]
    L.orc_keys.argtypes = [ctypes.c_void_p, _U64, _I64]
    L.orc_cells.argtypes = [ctypes.c_void_p, _I32]
    L.orc_lists.argtypes = [ctypes.c_void_p, _I32, _I32, _I32, _I32]
    L.orc_evaluate.argtypes = [ctypes.c_void_p, _D, _D, ctypes.c_int, ctypes.c_int64, _I64, _D, _D]
    L.orc_expansions.argtypes = [ctypes.c_void_p, _D, _D]
    L.orc_backward.argtypes = [ctypes.c_void_p, _D, _D, _D, _D]
    L.orc_direct.argtypes = [_D, ctypes.c_int64, ctypes.c_int64, _I64, _D, _D]
    L.orc_op_p2m.argtypes = [ctypes.c_int, _D, ctypes.c_int, _D, _D]
    for name in ("orc_op_m2m", "orc_op_m2l", "orc_op_l2l", "orc_op_l2p", "orc_op_m2p"):
        getattr(L, name).argtypes = [ctypes.c_int, _D, _D, _D, _D]
    L.orc_harmonics.argtypes = [ctypes.c_int, _D, _D, _D]
    return L


def set_threads(n: int = 0) -> int:
    """Set the OpenMP thread count (0 = leave); returns the count in use."""
    return int(lib().orc_set_threads(int(n)))


def _dp(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _cplx_view(a: np.ndarray) -> np.ndarray:
    return a.view(np.complex128)


class OracleTree:
    """Tree, lists and evaluation of the oracle for one particle set.

    xyzq: (N, 4) array of x, y, z, q (any float dtype, widened to double).
    circumscribed / tight: the MAC radius (half diagonal; distance from the
    cube centre to the farthest body).  fitted: expansion centres at the
    centre of the box of the cell's bodies (their voxel centres), the MAC
    radius the distance from there to the farthest body.
    """

    def __init__(self, xyzq, p: int, theta: float, ncrit: int, circumscribed: bool = False,
                 tight: bool = False, fitted: bool = False):
        L = lib()
        self.xyzq = _f64(xyzq).reshape(-1, 4)
        self.N = self.xyzq.shape[0]
        self.p = int(p)
        h = ctypes.c_void_p()
        rc = L.orc_build(_dp(self.xyzq), self.N, self.p, float(theta), int(ncrit),
                         (1 if circumscribed else 0) | (2 if tight else 0) | (4 if fitted else 0),
                         ctypes.byref(h))
        if rc != 0:
            raise ValueError(f"oracle build failed with code {rc}")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().orc_free(h)
            self._h = None

    def centres(self) -> np.ndarray:
        """Expansion centre of every cell, (ncell, 3)."""
        out = np.zeros((self.info()["ncell"], 3))
        lib().orc_centres(self._h, _dp(out))
        return out

    def set_order(self, p: int) -> None:
        """Evaluate with p terms from now on (same tree and lists)."""
        if lib().orc_set_order(self._h, int(p)) != 0:
            raise ValueError(f"bad order {p}")
        self.p = int(p)

    def info(self) -> dict:
        out = np.zeros(6, np.int64)
        lib().orc_info(self._h, out.ctypes.data_as(_I64))
        keys = ("ncell", "nleaf", "nlevel", "n_p2p", "n_m2l", "p2p_pairs")
        return {k: int(v) for k, v in zip(keys, out)}

    def root(self) -> dict:
        out = np.zeros(13)
        lib().orc_root(self._h, _dp(out))
        return {"lo": out[0:3], "hi": out[3:6], "centre": out[6:9], "H": out[9], "corner": out[10:13]}

    def keys(self):
        k = np.zeros(self.N, np.uint64)
        perm = np.zeros(self.N, np.int64)
        lib().orc_keys(self._h, k.ctypes.data_as(_U64), perm.ctypes.data_as(_I64))
        return k, perm

    def cells(self) -> dict:
        n = self.info()["ncell"]
        out = np.zeros((9, n), np.int32)
        lib().orc_cells(self._h, out.ctypes.data_as(_I32))
        names = ("level", "ix", "iy", "iz", "body_begin", "body_end", "child_begin",
                 "child_count", "parent")
        return {k: out[i] for i, k in enumerate(names)}

    def lists(self) -> dict:
        inf = self.info()
        a = [np.zeros(inf["n_p2p"], np.int32) for _ in range(2)]
        b = [np.zeros(inf["n_m2l"], np.int32) for _ in range(2)]
        lib().orc_lists(self._h, *(x.ctypes.data_as(_I32) for x in a + b))
        return {"p2p_tgt": a[0], "p2p_src": a[1], "m2l_tgt": b[0], "m2l_src": b[1]}

    def evaluate(self, q=None, xyz=None, mode: int = 3, targets=None):
        """Returns (phi, grad) in input order, or in the order of `targets`."""
        qq = None if q is None else _f64(q).reshape(-1)
        xx = None if xyz is None else _f64(xyz).reshape(-1, 3)
        tt = None if targets is None else np.ascontiguousarray(np.asarray(targets, np.int64))
        nt = self.N if tt is None else tt.shape[0]
        phi = np.zeros(nt)
        grad = np.zeros((nt, 3))
        rc = lib().orc_evaluate(self._h, _dp(xx), _dp(qq), int(mode), nt,
                                None if tt is None else tt.ctypes.data_as(_I64), _dp(phi), _dp(grad))
        if rc != 0:
            raise ValueError(f"oracle evaluate failed with code {rc}")
        return phi, grad

    def expansions(self):
        """(M, L) of the last evaluation, complex arrays of shape (ncell, p*p)."""
        n = self.info()["ncell"]
        M = np.zeros((n, self.p * self.p * 2))
        Lc = np.zeros((n, self.p * self.p * 2))
        lib().orc_expansions(self._h, _dp(M), _dp(Lc))
        return _cplx_view(M), _cplx_view(Lc)

    def backward(self, w, q=None):
        """Adjoint of sum_i w_i phi_i: returns (dL/dq, dL/dx)."""
        ww = _f64(w).reshape(-1)
        qq = None if q is None else _f64(q).reshape(-1)
        dq = np.zeros(self.N)
        dx = np.zeros((self.N, 3))
        rc = lib().orc_backward(self._h, _dp(qq), _dp(ww), _dp(dq), _dp(dx))
        if rc != 0:
            raise ValueError(f"oracle backward failed with code {rc}")
        return dq, dx


def direct(xyzq, targets=None):
    """Direct double-precision sum: (phi, grad) at the targets (input indices)."""
    a = _f64(xyzq).reshape(-1, 4)
    tt = None if targets is None else np.ascontiguousarray(np.asarray(targets, np.int64))
    nt = a.shape[0] if tt is None else tt.shape[0]
    phi = np.zeros(nt)
    grad = np.zeros((nt, 3))
    lib().orc_direct(_dp(a), a.shape[0], nt, None if tt is None else tt.ctypes.data_as(_I64),
                     _dp(phi), _dp(grad))
    return phi, grad


# ---- single operators, complex arrays of p*p entries (index n*(n+1)+m)

def _cz(p):
    return np.zeros(p * p, np.complex128)


def p2m(p, centre, xyzq):
    a = _f64(xyzq).reshape(-1, 4)
    M = _cz(p)
    lib().orc_op_p2m(p, _dp(_f64(centre)), a.shape[0], _dp(a), M.view(np.float64).ctypes.data_as(_D))
    return M


def _op(name, p, X, c1, c2, out=None):
    X = np.ascontiguousarray(X, np.complex128)
    out = _cz(p) if out is None else out
    getattr(lib(), name)(p, X.view(np.float64).ctypes.data_as(_D), _dp(_f64(c1)), _dp(_f64(c2)),
                         out.view(np.float64).ctypes.data_as(_D))
    return out


def m2m(p, Mc, c_child, c_parent):
    return _op("orc_op_m2m", p, Mc, c_child, c_parent)


def m2l(p, M, c_src, c_tgt):
    return _op("orc_op_m2l", p, M, c_src, c_tgt)


def l2l(p, Lp, c_parent, c_child):
    return _op("orc_op_l2l", p, Lp, c_parent, c_child)


def _eval(name, p, X, c, x):
    X = np.ascontiguousarray(X, np.complex128)
    out = np.zeros(4)
    getattr(lib(), name)(p, X.view(np.float64).ctypes.data_as(_D), _dp(_f64(c)), _dp(_f64(x)), _dp(out))
    return out[0], out[1:4].copy()


def l2p(p, L, c, x):
    """(phi, grad) of a local expansion at x."""
    return _eval("orc_op_l2p", p, L, c, x)


def m2p(p, M, c, x):
    """(phi, grad) of a multipole expansion at x."""
    return _eval("orc_op_m2p", p, M, c, x)


def harmonics(p, v):
    U = _cz(p)
    T = _cz(p)
    lib().orc_harmonics(p, _dp(_f64(v)), U.view(np.float64).ctypes.data_as(_D),
                        T.view(np.float64).ctypes.data_as(_D))
    return U, T
