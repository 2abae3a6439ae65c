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


# Per-body bound next to the relative L2 tolerance: the largest error of one
# body (the vector error for forces) relative to the largest reference value.
# It catches a few bad bodies that a norm over a million would hide.
TOL_BODY_PHI, TOL_BODY_F = 1e-4, 1e-3


def max_body_err(a, b):
    """max_i |a_i - b_i| / max_i |b_i|; rows are compared as vectors."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if a.ndim == 2:
        d, r = np.linalg.norm(a - b, axis=1), np.linalg.norm(b, axis=1)
    else:
        d, r = np.abs(a - b), np.abs(b)
    return float(d.max() / r.max())


def assert_match(phi, phi_ref, f, f_ref, tol_phi, tol_f, body_phi=TOL_BODY_PHI, body_f=TOL_BODY_F):
    """Relative L2 within the tolerances, and every body within the
    per-body bounds."""
    e = (rel(phi, phi_ref), rel(f, f_ref), max_body_err(phi, phi_ref), max_body_err(f, f_ref))
    assert e[0] < tol_phi and e[1] < tol_f, e
    assert e[2] < body_phi and e[3] < body_f, e
    return e
