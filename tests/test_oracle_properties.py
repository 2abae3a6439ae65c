"""Property tests of the oracle on small generated body sets, including
degenerate geometry: bodies on a line or a plane, repeated points, clusters
far apart, and coordinates of very large or very small magnitude. For every
set: the root cube, keys, order and cells equal their definitions written out
with plain integers, every (target, source) body pair is covered exactly once
by P2P or by one M2L, the lists are symmetric, every cell's bodies lie in its
cube, with the MAC switched off (theta tiny) the result is the direct sum, the
operator is symmetric, and the result equals the independent Cartesian Taylor
checker. With the circumscribed radius, every body's potential error stays
under the sum, over the M2L pairs that reach it, of the double-truncation
bound Q_A rho^p / (d - r_A - r_B), rho = (r_A + r_B) / d: M2M and L2L are
exact within the degree < p truncation, so the M2L truncations are the only
error.
"""

import numpy as np
import pytest

from tests.test_oracle_pins import _fitted_geometry

hyp = pytest.importorskip("hypothesis")
from hypothesis import HealthCheck, given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402


# The expansions use unscaled solid harmonics (r^n and 1/r^(n+1) up to degree
# 2p - 2), so the far field needs cell sizes whose powers stay inside the double
# range; the tree, the lists and the near field have no such limit.
ALL_SCALES = (1e-30, 1e-6, 1.0, 1e6, 1e30)
FAR_FIELD_SCALES = (1e-12, 1e-6, 1.0, 1e6, 1e12)


@st.composite
def body_sets(draw, scales=ALL_SCALES):
    n = draw(st.integers(1, 160))
    seed = draw(st.integers(0, 2 ** 31 - 1))
    shape = draw(st.sampled_from(["cube", "line", "plane", "repeats", "clusters"]))
    scale = draw(st.sampled_from(scales))
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, (n, 3))
    if shape == "line":
        x = np.outer(rng.uniform(-1, 1, n), rng.normal(size=3))
    elif shape == "plane":
        x[:, draw(st.integers(0, 2))] = 0.25
    elif shape == "repeats":
        x = x[rng.integers(0, max(1, n // 4), n)]
    elif shape == "clusters":
        x = 1e-3 * x + np.where(rng.random((n, 1)) < 0.5, -1.0, 1.0) * np.array([1.0, 0.5, 0.25])
    q = rng.uniform(-1, 1, n)
    return np.concatenate([scale * x, q[:, None]], axis=1)


def _covered_once(T, n):
    c = T.cells()
    L = T.lists()
    bb, be = c["body_begin"], c["body_end"]
    cnt = np.zeros((n, n), np.int32)
    for t, s in zip(L["p2p_tgt"], L["p2p_src"]):
        cnt[bb[t]:be[t], bb[s]:be[s]] += 1
    for t, s in zip(L["m2l_tgt"], L["m2l_src"]):
        cnt[bb[t]:be[t], bb[s]:be[s]] += 1
    assert np.all(cnt == 1)
    for a, b in (("p2p_tgt", "p2p_src"), ("m2l_tgt", "m2l_src")):
        pairs = set(zip(L[a].tolist(), L[b].tolist()))
        assert all((s, t) in pairs for t, s in pairs)


def _bodies_in_cells(T, x):
    c = T.cells()
    r = T.root()
    _, perm = T.keys()
    xs = x[perm, :3]
    for i in range(c["level"].size):
        R = np.ldexp(r["H"], -int(c["level"][i]))
        lo = r["corner"] + 2 * R * np.array([c["ix"][i], c["iy"][i], c["iz"][i]], np.float64)
        b = xs[c["body_begin"][i]:c["body_end"][i]]
        tol = 1e-12 * r["H"]
        assert np.all(b >= lo - tol) and np.all(b <= lo + 2 * R + tol)


@settings(max_examples=300, deadline=None, derandomize=True, suppress_health_check=[HealthCheck.too_slow])
@given(x=body_sets(), ncrit=st.integers(1, 12), theta=st.sampled_from([0.3, 0.5, 0.7, 0.95]),
       mode=st.sampled_from(["half", "circumscribed", "tight", "fitted"]))
def test_traversal_covers_every_pair_once(orc, x, ncrit, theta, mode):
    T = _tree(orc, x, 3, theta, ncrit, mode)
    _covered_once(T, x.shape[0])
    _bodies_in_cells(T, x)


@settings(max_examples=200, deadline=None, derandomize=True, suppress_health_check=[HealthCheck.too_slow])
@given(x=body_sets(), ncrit=st.integers(1, 12))
def test_no_acceptance_gives_the_direct_sum(orc, x, ncrit):
    T = orc.OracleTree(x, 2, 1e-9, ncrit)
    assert T.info()["n_m2l"] == 0
    ph, g = T.evaluate()
    pd, gd = orc.direct(x)
    np.testing.assert_allclose(ph, pd, rtol=1e-12, atol=1e-12 * np.abs(pd).max(initial=0))
    np.testing.assert_allclose(g, gd, rtol=1e-12, atol=1e-12 * np.abs(gd).max(initial=0))


@settings(max_examples=200, deadline=None, derandomize=True, suppress_health_check=[HealthCheck.too_slow])
@given(x=body_sets(FAR_FIELD_SCALES), ncrit=st.integers(1, 12), theta=st.sampled_from([0.3, 0.5, 0.7]),
       p=st.integers(1, 7))
def test_potential_error_within_the_truncation_bound(orc, x, ncrit, theta, p):
    T = orc.OracleTree(x, p, theta, ncrit, circumscribed=True)
    c = T.cells()
    L = T.lists()
    r = T.root()
    _, perm = T.keys()
    bb, be = c["body_begin"], c["body_end"]
    R = np.ldexp(r["H"], -c["level"].astype(np.int64))
    ctr = r["corner"] + R[:, None] * (2.0 * np.stack([c["ix"], c["iy"], c["iz"]], 1) + 1.0)
    rad = np.sqrt(3.0) * R
    qa = np.abs(x[perm, 3])
    Q = np.array([qa[bb[i]:be[i]].sum() for i in range(R.size)])
    bound = np.zeros(x.shape[0])
    for t, s in zip(L["m2l_tgt"], L["m2l_src"]):
        d = np.linalg.norm(ctr[t] - ctr[s])
        rho = (rad[t] + rad[s]) / d
        assert rho < theta * (1 + 1e-12)
        bound[bb[t]:be[t]] += Q[s] * rho ** p / (d - rad[t] - rad[s])
    ph, _ = T.evaluate()
    pd, _ = orc.direct(x)
    absq = x.copy()
    absq[:, 3] = np.abs(absq[:, 3])
    scale, _ = orc.direct(absq)  # sum_j |q_j| / r_ij: the size of the rounding errors
    err = np.abs(ph - pd)[perm]
    assert np.all(err <= bound * (1 + 1e-9) + 1e-12 * scale[perm])


@settings(max_examples=150, deadline=None, derandomize=True, suppress_health_check=[HealthCheck.too_slow])
@given(x=body_sets(FAR_FIELD_SCALES), ncrit=st.integers(1, 12), theta=st.sampled_from([0.3, 0.5, 0.7]),
       p=st.integers(1, 7), mode=st.sampled_from(["half", "circumscribed", "tight", "fitted"]),
       wseed=st.integers(0, 2 ** 31 - 1))
def test_operator_is_symmetric(orc, x, ncrit, theta, p, mode, wseed):
    """The truncated kernel of an M2L pair is a polynomial of degree < p in each
    of the two offsets with the coefficients of the even 1/r, and the lists are
    symmetric, so the FMM operator is symmetric: w . FMM(q) = q . FMM(w)."""
    T = _tree(orc, x, p, theta, ncrit, mode)
    q = x[:, 3]
    w = np.random.default_rng(wseed).uniform(-1, 1, x.shape[0])
    pq, _ = T.evaluate(q)
    pw, _ = T.evaluate(w)
    absx = x.copy()
    absx[:, 3] = 1.0
    s, _ = orc.direct(absx)  # sum_j 1 / r_ij: the size of the terms
    size = float(np.abs(w) @ (s * np.abs(q).max())) + float(np.abs(q) @ (s * np.abs(w).max()))
    assert abs(float(w @ pq) - float(q @ pw)) <= 1e-11 * size + 1e-300


@settings(max_examples=60, deadline=None, derandomize=True, suppress_health_check=[HealthCheck.too_slow])
@given(x=body_sets((1e-3, 1.0, 1e3)), ncrit=st.integers(1, 8), theta=st.sampled_from([0.5, 0.7]),
       p=st.integers(1, 4), mode=st.sampled_from(["half", "circumscribed", "tight", "fitted"]))
def test_matches_the_cartesian_checker(orc, x, ncrit, theta, p, mode):
    """The whole oracle equals the basis-free double Taylor closed form of the
    same lists (an independent Cartesian evaluation with no M2M or L2L)."""
    from tests import taylor_checker
    x = x[:60]
    T = _tree(orc, x, p, theta, ncrit, mode)
    ph, g = T.evaluate()
    # fitted: the centres derived from the bodies' voxel coordinates, not read
    # from the oracle
    centres = _fitted_geometry(T)[2] if mode == "fitted" else None
    ph2, g2 = taylor_checker.evaluate(x, p, T.cells(), T.lists(), T.keys(), T.root(), centres=centres)
    # sizes of the summed terms, sum_j |q_j| / r_ij and sum_j |q_j| / r_ij^2,
    # set the rounding tolerance
    d = np.linalg.norm(x[:, None, :3] - x[None, :, :3], axis=2)
    inv = np.divide(1.0, d, out=np.zeros_like(d), where=d > 0)
    s1 = inv @ np.abs(x[:, 3])
    s2 = (inv * inv) @ np.abs(x[:, 3])
    assert np.all(np.abs(ph - ph2) <= 1e-11 * s1)
    assert np.all(np.abs(g - g2).max(1) <= 1e-10 * s2)


def _tree(orc, x, p, theta, ncrit, mode):
    return orc.OracleTree(x, p, theta, ncrit, circumscribed=mode == "circumscribed", tight=mode == "tight",
                          fitted=mode == "fitted")


def _brute_tree(x, ncrit):
    """Root cube, keys, order and cells written out from their definitions
    (Sec. II.B/II.C, Sec. III.A's N_crit) with plain Python integers."""
    lo, hi = x[:, :3].min(0), x[:, :3].max(0)
    ctr = (lo + hi) * 0.5
    H = max(float(v) for v in (hi - lo) * 0.5) * (1.0 + 2.0 ** -20)
    H = 0.5 if H == 0.0 else H
    corner = ctr - H
    per_len = 2.0 ** 21 / (2.0 * H)  # voxels per unit length, rounded once
    k = np.floor((x[:, :3] - corner) * per_len)
    k = np.clip(k, 0, 2 ** 21 - 1).astype(np.int64)
    keys = []
    for kx, ky, kz in k.tolist():
        key = 0
        for b in range(21):  # x is the most significant bit of each triple
            key |= (((kx >> b) & 1) << (3 * b + 2)) | (((ky >> b) & 1) << (3 * b + 1)) | (((kz >> b) & 1) << (3 * b))
        keys.append(key)
    perm = sorted(range(len(keys)), key=lambda i: (keys[i], i))
    ks = [keys[i] for i in perm]
    # breadth-first cells: (level, prefix, begin, end, parent)
    cells = [(0, 0, 0, len(ks), -1)]
    child_begin, child_count = [], []
    i = 0
    while i < len(cells):
        lev, pre, b, e, _ = cells[i]
        if e - b > ncrit and lev < 21:
            first = len(cells)
            shift = 3 * (21 - lev - 1)
            j = b
            while j < e:
                pc = ks[j] >> shift
                m = j
                while m < e and ks[m] >> shift == pc:
                    m += 1
                cells.append((lev + 1, pc, j, m, i))
                j = m
            child_begin.append(first)
            child_count.append(len(cells) - first)
        else:
            child_begin.append(-1)
            child_count.append(0)
        i += 1

    def coord(pre, lev, axis_bit):
        v = 0
        for b in range(lev):
            v |= ((pre >> (3 * b + axis_bit)) & 1) << b
        return v

    out = {"level": [c[0] for c in cells],
           "ix": [coord(c[1], c[0], 2) for c in cells], "iy": [coord(c[1], c[0], 1) for c in cells],
           "iz": [coord(c[1], c[0], 0) for c in cells],
           "body_begin": [c[2] for c in cells], "body_end": [c[3] for c in cells],
           "child_begin": child_begin, "child_count": child_count, "parent": [c[4] for c in cells]}
    return {"lo": lo, "hi": hi, "centre": ctr, "H": H, "corner": corner}, ks, perm, out


@settings(max_examples=200, deadline=None, derandomize=True, suppress_health_check=[HealthCheck.too_slow])
@given(x=body_sets(), ncrit=st.integers(1, 12))
def test_tree_equals_its_definition(orc, x, ncrit):
    T = orc.OracleTree(x, 2, 0.5, ncrit)
    root, ks, perm, cells = _brute_tree(x.astype(np.float64), ncrit)
    r = T.root()
    for name in ("lo", "hi", "centre", "corner"):
        assert np.array_equal(r[name], root[name]), name
    assert r["H"] == root["H"]
    keys, operm = T.keys()
    assert keys.tolist() == ks and operm.tolist() == perm
    c = T.cells()
    for name, v in cells.items():
        assert c[name].tolist() == v, name
