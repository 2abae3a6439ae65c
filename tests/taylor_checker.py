"""Independent Cartesian-Taylor evaluation of the FMM approximant (test helper).

The FMM with degree-< p multipole and local expansions and exact M2M/L2L
translations computes, for a target x_i in cell B and a source y_j in a cell
A with an M2L pair (A -> B) on the path of x_i's leaf, the double Taylor
truncation of 1/|x - y| about (c_B, c_A):

    sum_{|alpha| < p, |beta| < p}  d^(alpha+beta)(1/r)(c_B - c_A)
                                   * a^alpha (-b)^beta / (alpha! beta!),

with a = x_i - c_B and b = y_j - c_A (the degree-n term of a solid-harmonic
expansion is the degree-n homogeneous part of the Taylor series, so the basis
does not matter).  This module evaluates that closed form with Cartesian
monomials and no M2M, L2L or spherical harmonics, so it pins the oracle's
normalisation and sign conventions independently.

The Taylor coefficients t_g = d^g(1/r)(D)/g! come from the ray recurrence:
along h = s v, G(s) = (|D|^2 + 2 s D.v + s^2 |v|^2)^(-1/2) solves
(|D|^2 + 2 s D.v + s^2 |v|^2) G' = -(D.v + s |v|^2) G, whose Taylor
coefficients give, for |g| = n >= 1,
    n |D|^2 t_g + (2n - 1) sum_i D_i t_(g - e_i) + (n - 1) sum_i t_(g - 2 e_i) = 0.
"""

from __future__ import annotations

from functools import lru_cache
from math import factorial

import numpy as np


@lru_cache(maxsize=None)
def multi_indices(order: int):
    """All (gx, gy, gz) with gx + gy + gz <= order, grouped by total degree."""
    out = []
    for n in range(order + 1):
        for gx in range(n, -1, -1):
            for gy in range(n - gx, -1, -1):
                out.append((gx, gy, n - gx - gy))
    return tuple(out)


def taylor_coefficients(D, order: int) -> dict:
    """t_g = d^g (1/|.|)(D) / g! for |g| <= order."""
    D = np.asarray(D, dtype=np.float64)
    d2 = float(D @ D)
    t = {(0, 0, 0): 1.0 / np.sqrt(d2)}
    for g in multi_indices(order)[1:]:
        n = sum(g)
        s = 0.0
        for i in range(3):
            if g[i] >= 1:
                gm = list(g); gm[i] -= 1
                s += (2 * n - 1) * D[i] * t[tuple(gm)]
            if g[i] >= 2:
                gm = list(g); gm[i] -= 2
                s += (n - 1) * t[tuple(gm)]
        t[g] = -s / (n * d2)
    return t


def _fact3(g):
    return factorial(g[0]) * factorial(g[1]) * factorial(g[2])


def _powers(v: np.ndarray, idx) -> np.ndarray:
    """(len(v), len(idx)) array of monomials v^g."""
    return np.stack([v[:, 0] ** g[0] * v[:, 1] ** g[1] * v[:, 2] ** g[2] for g in idx], axis=1)


def m2l_pair(p: int, D, b: np.ndarray, q: np.ndarray, a: np.ndarray):
    """Far-field contribution of sources (offsets b from c_A, charges q) to
    targets (offsets a from c_B) with D = c_B - c_A: (phi, grad)."""
    idx = [g for g in multi_indices(p - 1)]
    t = taylor_coefficients(D, 2 * p - 2)
    # moments mu_beta = sum_j q_j (-b_j)^beta / beta!
    mu = (_powers(-b, idx) * q[:, None]).sum(axis=0) / np.array([_fact3(g) for g in idx])
    # lambda_alpha = sum_beta (alpha+beta)! t_(alpha+beta) mu_beta
    lam = np.zeros(len(idx))
    for ia, al in enumerate(idx):
        s = 0.0
        for ib, be in enumerate(idx):
            g = (al[0] + be[0], al[1] + be[1], al[2] + be[2])
            s += _fact3(g) * t[g] * mu[ib]
        lam[ia] = s
    inv_af = np.array([1.0 / _fact3(g) for g in idx])
    phi = _powers(a, idx) @ (lam * inv_af)
    grad = np.zeros((a.shape[0], 3))
    for k in range(3):
        dcoef = []
        didx = []
        for ia, al in enumerate(idx):
            if al[k] == 0:
                continue
            gm = list(al); gm[k] -= 1
            didx.append(tuple(gm))
            dcoef.append(lam[ia] * inv_af[ia] * al[k])
        if didx:
            grad[:, k] = _powers(a, didx) @ np.array(dcoef)
    return phi, grad


def evaluate(xyzq: np.ndarray, p: int, cells: dict, lists: dict, keys_perm, root: dict, centres=None):
    """(phi, grad) in input order from the oracle's tree and lists, using only
    direct P2P sums and per-pair Cartesian double-Taylor M2L.  centres: the
    expansion centre of every cell, (ncell, 3); default the cube centres."""
    xyzq = np.asarray(xyzq, np.float64)
    _, perm = keys_perm
    xs = xyzq[perm, :3]
    qs = xyzq[perm, 3]
    N = xs.shape[0]
    H = root["H"]
    r0 = root["corner"]
    lev = cells["level"]
    cen = np.stack([r0[i] + (2.0 * cells[k] + 1.0) * np.ldexp(H, -lev)
                    for i, k in enumerate(("ix", "iy", "iz"))], axis=1)
    if centres is not None:
        cen = np.asarray(centres, np.float64)
    bb, be = cells["body_begin"], cells["body_end"]
    phi = np.zeros(N)
    grad = np.zeros((N, 3))
    for tgt, src in zip(lists["m2l_tgt"], lists["m2l_src"]):
        a = xs[bb[tgt]:be[tgt]] - cen[tgt]
        b = xs[bb[src]:be[src]] - cen[src]
        ph, gr = m2l_pair(p, cen[tgt] - cen[src], b, qs[bb[src]:be[src]], a)
        phi[bb[tgt]:be[tgt]] += ph
        grad[bb[tgt]:be[tgt]] += gr
    for tgt, src in zip(lists["p2p_tgt"], lists["p2p_src"]):
        xt = xs[bb[tgt]:be[tgt]]
        ys = xs[bb[src]:be[src]]
        d = xt[:, None, :] - ys[None, :, :]
        r2 = (d * d).sum(-1)
        with np.errstate(divide="ignore"):
            inv = np.where(r2 > 0, 1.0 / np.sqrt(np.where(r2 > 0, r2, 1.0)), 0.0)
        qq = qs[bb[src]:be[src]][None, :]
        phi[bb[tgt]:be[tgt]] += (qq * inv).sum(1)
        grad[bb[tgt]:be[tgt]] -= ((qq * inv ** 3)[:, :, None] * d).sum(1)
    out_phi = np.zeros(N)
    out_grad = np.zeros((N, 3))
    out_phi[perm] = phi
    out_grad[perm] = grad
    return out_phi, out_grad
