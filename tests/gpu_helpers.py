"""Shared helpers of the GPU tests (conversion of the library's real-packed,
scaled expansions to the oracle's complex, unscaled ones; error norms)."""

import numpy as np


def rel(a, b):
    """Relative L2 error (complex arrays compare both parts)."""
    a = np.asarray(a)
    b = np.asarray(b)
    dt = np.complex128 if (np.iscomplexobj(a) or np.iscomplexobj(b)) else np.float64
    a = a.astype(dt)
    b = b.astype(dt)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def unpack(X: np.ndarray, p: int) -> np.ndarray:
    """Real packing (n*n, n*n + 2m - 1, n*n + 2m) -> full complex (n*(n+1)+m)."""
    out = np.zeros((X.shape[0], p * p), np.complex128)
    for n in range(p):
        out[:, n * (n + 1)] = X[:, n * n]
        for m in range(1, n + 1):
            v = X[:, n * n + 2 * m - 1] + 1j * X[:, n * n + 2 * m]
            out[:, n * (n + 1) + m] = v
            out[:, n * (n + 1) - m] = (-1) ** m * np.conj(v)
    return out


def degree_of_index(p: int) -> np.ndarray:
    d = np.zeros(p * p, np.int64)
    for n in range(p):
        d[n * n:(n + 1) * (n + 1)] = n
    return d


def scale_oracle(Mo: np.ndarray, Lo: np.ndarray, R: np.ndarray, p: int):
    """Oracle (unscaled) -> the library's scaling: M / R^n, L * R^(n+1)."""
    deg = degree_of_index(p)
    Ms = Mo / R[:, None] ** deg[None, :]
    Ls = Lo * R[:, None] ** (deg[None, :] + 1)
    return Ms, Ls
