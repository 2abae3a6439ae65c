"""Pins of the double-precision oracle against facts fixed outside it.

None of these re-types the oracle's formulas: each compares it with a closed
form, a library routine (SciPy's Legendre functions), the exact 1/r
(addition theorem), an exact algebraic identity, an independent Cartesian
Taylor evaluation, brute force, or an invariance of the mathematics.
"""

import math

import numpy as np
import pytest
from scipy.special import lpmv

from paper_1405_7487_gb300 import workloads as W
from tests import taylor_checker


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def hidx(n, m):
    return n * (n + 1) + m


# ----------------------------------------------------------- harmonics

def test_harmonics_against_scipy_legendre(orc):
    """Ups_n^m = r^n P_n^m(cos t) e^{im phi}/(n+m)!, Th_n^m = (n-m)! P_n^m e^{im phi}/r^{n+1}
    with SciPy's Condon-Shortley P_n^m (lpmv), for all n < 12, |m| <= n."""
    p = 12
    rng = np.random.default_rng(3)
    for _ in range(5):
        v = rng.uniform(-1.5, 1.5, 3)
        U, T = orc.harmonics(p, v)
        r = np.linalg.norm(v)
        ct = v[2] / r
        ph = math.atan2(v[1], v[0])
        for n in range(p):
            for m in range(-n, n + 1):
                am = abs(m)
                P = lpmv(am, n, ct)
                u = r ** n * P * np.exp(1j * am * ph) / math.factorial(n + am)
                t = math.factorial(n - am) * P * np.exp(1j * am * ph) / r ** (n + 1)
                if m < 0:
                    u = (-1) ** am * np.conj(u)
                    t = (-1) ** am * np.conj(t)
                assert abs(U[hidx(n, m)] - u) <= 1e-12 * max(1.0, abs(u))
                assert abs(T[hidx(n, m)] - t) <= 1e-12 * max(1e-300, abs(t)) + 1e-300


def test_harmonics_low_degree_closed_forms(orc):
    x, y, z = 0.3, -0.7, 1.1
    r2 = x * x + y * y + z * z
    r = math.sqrt(r2)
    U, T = orc.harmonics(3, [x, y, z])
    assert U[hidx(0, 0)] == 1.0
    assert np.isclose(U[hidx(1, 0)], z)
    assert np.isclose(U[hidx(1, 1)], -(x + 1j * y) / 2)
    assert np.isclose(U[hidx(2, 0)], (2 * z * z - x * x - y * y) / 4)
    assert np.isclose(T[hidx(0, 0)], 1 / r)
    assert np.isclose(T[hidx(1, 0)], z / r ** 3)
    assert np.isclose(T[hidx(1, 1)], -(x + 1j * y) / r ** 3)


# ---------------------------------------------------- single operators

def _cloud(rng, n, centre, radius):
    d = rng.normal(size=(n, 3))
    d *= (radius * rng.random(n) ** (1 / 3) / np.linalg.norm(d, axis=1))[:, None]
    q = rng.uniform(-1, 1, n)
    return np.concatenate([centre + d, q[:, None]], axis=1)


def _direct_at(src, x):
    d = x[None, :] - src[:, :3]
    r = np.linalg.norm(d, axis=1)
    phi = (src[:, 3] / r).sum()
    grad = -((src[:, 3] / r ** 3)[:, None] * d).sum(0)
    return phi, grad


def test_addition_theorem_p30(orc):
    """P2M -> M2L -> L2P of a source cloud equals 1/r and its gradient to 1e-13 at p=30,
    and P2M -> M2P equals them too."""
    rng = np.random.default_rng(5)
    p = 30
    cA = np.array([0.1, -0.2, 0.05])
    cB = cA + np.array([1.0, 0.8, -0.6])
    src = _cloud(rng, 20, cA, 0.15)
    M = orc.p2m(p, cA, src)
    L = orc.m2l(p, M, cA, cB)
    for x in _cloud(rng, 10, cB, 0.15)[:, :3]:
        ph_d, g_d = _direct_at(src, x)
        ph, g = orc.l2p(p, L, cB, x)
        assert abs(ph - ph_d) <= 1e-13 * abs(src[:, 3]).sum()
        assert np.linalg.norm(g - g_d) <= 1e-12 * np.linalg.norm(g_d)
        ph2, g2 = orc.m2p(p, M, cA, x)
        assert abs(ph2 - ph_d) <= 1e-13 * abs(src[:, 3]).sum()
        assert np.linalg.norm(g2 - g_d) <= 1e-12 * np.linalg.norm(g_d)


def test_single_interaction_error_bound(orc):
    """|error| of the double truncation stays below
    Q/(d - ra - rb) * ((ra + rb)/d)^p for every p (Q = sum |q|)."""
    rng = np.random.default_rng(11)
    for trial in range(20):
        ra, rb = rng.uniform(0.1, 0.4, 2)
        d = (ra + rb) / rng.uniform(0.3, 0.7)
        u = rng.normal(size=3); u /= np.linalg.norm(u)
        cA = rng.uniform(-1, 1, 3)
        cB = cA + d * u
        src = _cloud(rng, 8, cA, ra)
        Q = np.abs(src[:, 3]).sum()
        x = _cloud(rng, 1, cB, rb)[0, :3]
        ph_d, _ = _direct_at(src, x)
        for p in (2, 4, 6, 8, 12):
            M = orc.p2m(p, cA, src)
            ph, _ = orc.l2p(p, orc.m2l(p, M, cA, cB), cB, x)
            bound = Q / (d - ra - rb) * ((ra + rb) / d) ** p
            assert abs(ph - ph_d) <= bound * (1 + 1e-9) + 1e-14


def test_m2m_exact(orc):
    """M2M of P2M(child bodies) equals P2M of the same bodies about the parent."""
    rng = np.random.default_rng(7)
    p = 12
    cp = np.array([0.5, 0.5, 0.5])
    Mp = np.zeros(p * p, np.complex128)
    allb = []
    for o in range(8):
        off = np.array([(o >> 2) & 1, (o >> 1) & 1, o & 1]) - 0.5
        cc = cp + 0.25 * off
        b = _cloud(rng, 7, cc, 0.2)
        allb.append(b)
        Mc = orc.p2m(p, cc, b)
        Mp += orc.m2m(p, Mc, cc, cp)
    ref = orc.p2m(p, cp, np.concatenate(allb))
    assert np.max(np.abs(Mp - ref)) <= 1e-14 * np.max(np.abs(ref)) * 10


def test_l2l_exact(orc):
    """L2P(L2L(L)) equals L2P(L) (a degree < p polynomial shifts exactly)."""
    rng = np.random.default_rng(8)
    p = 10
    cP = np.zeros(3)
    L = (rng.normal(size=p * p) + 1j * rng.normal(size=p * p))
    # make it the expansion of a real field: L_n^{-m} = (-1)^m conj(L_n^m)
    for n in range(p):
        L[hidx(n, 0)] = L[hidx(n, 0)].real
        for m in range(1, n + 1):
            L[hidx(n, -m)] = (-1) ** m * np.conj(L[hidx(n, m)])
    cC = np.array([0.25, -0.25, 0.25])
    Lc = orc.l2l(p, L, cP, cC)
    for x in rng.uniform(-0.25, 0.25, (5, 3)) + cC:
        a = orc.l2p(p, L, cP, x)
        b = orc.l2p(p, Lc, cC, x)
        assert abs(a[0] - b[0]) <= 1e-13 * max(1, abs(a[0]))
        assert np.linalg.norm(a[1] - b[1]) <= 1e-12 * max(1, np.linalg.norm(a[1]))


def test_l2p_gradient_matches_finite_difference(orc):
    rng = np.random.default_rng(9)
    p = 8
    src = _cloud(rng, 10, np.zeros(3), 0.2)
    cB = np.array([1.0, 0.4, -0.3])
    L = orc.m2l(p, orc.p2m(p, np.zeros(3), src), np.zeros(3), cB)
    x = cB + np.array([0.05, -0.1, 0.07])
    _, g = orc.l2p(p, L, cB, x)
    h = 1e-6
    fd = [(orc.l2p(p, L, cB, x + h * e)[0] - orc.l2p(p, L, cB, x - h * e)[0]) / (2 * h)
          for e in np.eye(3)]
    assert np.allclose(g, fd, rtol=1e-7, atol=1e-9)


# ---------------------------------------------------------- whole FMM

def test_all_p2p_when_root_is_a_leaf(orc):
    """ncrit >= N: the root is a leaf, everything is P2P, result == direct sum."""
    x = W.cube(500, 21)
    T = orc.OracleTree(x, 6, 0.4, 1000)
    assert T.info()["ncell"] == 1 and T.info()["n_m2l"] == 0
    ph, g = T.evaluate()
    pd, gd = orc.direct(x)
    assert rel(ph, pd) < 1e-13 and rel(g, gd) < 1e-13


def test_all_p2p_when_mac_never_accepts(orc):
    """theta tiny: no pair passes the MAC, so the traversal must reach every
    leaf pair and the result equals the direct sum."""
    x = W.cube(3000, 22)
    T = orc.OracleTree(x, 4, 0.01, 16)
    inf = T.info()
    assert inf["n_m2l"] == 0 and inf["nlevel"] >= 4
    ph, g = T.evaluate()
    pd, gd = orc.direct(x)
    assert rel(ph, pd) < 1e-13 and rel(g, gd) < 1e-13


@pytest.mark.parametrize("dist,p,theta,ncrit", [("cube", 3, 0.5, 16), ("cube", 5, 0.4, 24),
                                                ("plummer", 4, 0.5, 12)])
def test_matches_cartesian_taylor_checker(orc, dist, p, theta, ncrit):
    """The whole oracle equals the basis-free double Taylor closed form."""
    x = W.cube(600, 31) if dist == "cube" else W.plummer(600, 32)
    T = orc.OracleTree(x, p, theta, ncrit)
    assert T.info()["n_m2l"] > 0
    ph, g = T.evaluate()
    ph2, g2 = taylor_checker.evaluate(x, p, T.cells(), T.lists(), T.keys(), T.root())
    assert rel(ph, ph2) < 1e-12
    assert rel(g, g2) < 1e-11


def test_error_decreases_with_p(orc):
    x = W.cube(4096, 1)
    pd, gd = orc.direct(x)
    errs = []
    for p in range(2, 17):
        T = orc.OracleTree(x, p, 0.4, 64)
        ph, g = T.evaluate()
        errs.append((rel(ph, pd), rel(g, gd)))
    e = np.array(errs)
    assert np.all(np.diff(e[:, 0]) < 0) and np.all(np.diff(e[:, 1]) < 0)
    assert e[-1, 0] < 1e-8


def test_error_scales_like_theta_to_the_p_circumscribed(orc):
    """With the circumscribed radius the error behaves like C theta^p (Sec. III.A)."""
    x = W.cube(4096, 1)
    pd, _ = orc.direct(x)
    ps = np.arange(3, 12)
    e = []
    for p in ps:
        T = orc.OracleTree(x, int(p), 0.5, 64, circumscribed=True)
        e.append(rel(T.evaluate()[0], pd))
    slope = np.polyfit(ps, np.log(e), 1)[0]
    assert np.exp(slope) < 0.5 * 1.05  # decays at least like theta^p


# ---------------------------------------------------------- tree, lists

def test_tree_structure(orc):
    for x, ncrit in ((W.cube(5000, 41), 32), (W.plummer(5000, 42), 10)):
        T = orc.OracleTree(x, 4, 0.5, ncrit)
        keys, perm = T.keys()
        assert np.all(np.diff(keys.astype(np.int64)) >= 0)
        assert sorted(perm.tolist()) == list(range(len(perm)))
        c = T.cells()
        r = T.root()
        lev = c["level"]
        R = np.ldexp(r["H"], -lev)
        xs = np.asarray(x, np.float64)[perm]
        leaf = c["child_count"] == 0
        for i in np.nonzero(leaf)[0]:
            b = xs[c["body_begin"][i]:c["body_end"][i], :3]
            lo = r["corner"] + 2 * R[i] * np.array([c["ix"][i], c["iy"][i], c["iz"][i]])
            assert np.all(b >= lo - 1e-12) and np.all(b <= lo + 2 * R[i] + 1e-12)
            assert c["body_end"][i] - c["body_begin"][i] <= ncrit or lev[i] == 21
        split = ~leaf
        assert np.all(c["body_end"][split] - c["body_begin"][split] > ncrit)
        # leaves tile the body range
        bb = np.sort(c["body_begin"][leaf])
        assert bb[0] == 0 and np.all(np.diff(np.sort(c["body_end"][leaf])) > 0)


def test_traversal_covers_every_pair_exactly_once(orc):
    """Every (target body, source body) pair is covered once: by P2P between
    leaves or by one M2L into an ancestor-or-self of the target's leaf.
    All M2L pairs satisfy the MAC and the directed lists are symmetric."""
    x = W.plummer(1500, 51)
    T = orc.OracleTree(x, 4, 0.6, 8)
    c = T.cells()
    L = T.lists()
    N = x.shape[0]
    cnt = np.zeros((N, N), np.int32)
    bb, be = c["body_begin"], c["body_end"]
    for t, s in zip(L["p2p_tgt"], L["p2p_src"]):
        assert c["child_count"][t] == 0 and c["child_count"][s] == 0
        cnt[bb[t]:be[t], bb[s]:be[s]] += 1
    for t, s in zip(L["m2l_tgt"], L["m2l_src"]):
        cnt[bb[t]:be[t], bb[s]:be[s]] += 1
    assert np.all(cnt == 1)
    m2l = set(zip(L["m2l_tgt"].tolist(), L["m2l_src"].tolist()))
    assert all((s, t) in m2l for t, s in m2l)
    p2p = set(zip(L["p2p_tgt"].tolist(), L["p2p_src"].tolist()))
    assert all((s, t) in p2p for t, s in p2p)
    R = c["level"]
    # the larger cell is the one split (Dehnen): two non-leaves meeting in an
    # M2L differ by at most one level
    leaf = c["child_count"] == 0
    for t, s in m2l:
        if not leaf[t] and not leaf[s]:
            assert abs(int(R[t]) - int(R[s])) <= 1
    for t, s in m2l:
        ct = (2 * np.array([c["ix"][t], c["iy"][t], c["iz"][t]], np.int64) + 1) << (21 - R[t])
        cs = (2 * np.array([c["ix"][s], c["iy"][s], c["iz"][s]], np.int64) + 1) << (21 - R[s])
        d = np.sqrt(float(((ct - cs) ** 2).sum()))
        assert 0.6 * d > (1 << (21 - R[t])) + (1 << (21 - R[s]))


def test_tight_mac_covers_every_pair_once_and_bounds_hold(orc):
    """Particle-fitted MAC radius about the cube centre (Sec. II.B's tight
    bound): every body pair is still covered exactly once, and every M2L pair
    satisfies theta |c_A - c_B| > r_A + r_B, r the true distance from the
    centre to the farthest body (up to the voxel quantisation of the radii)."""
    x = W.plummer(1500, 52)
    theta = 0.6
    T = orc.OracleTree(x, 4, theta, 8, tight=True)
    c = T.cells()
    L = T.lists()
    r = T.root()
    N = x.shape[0]
    bb, be = c["body_begin"], c["body_end"]
    cnt = np.zeros((N, N), np.int32)
    for t, s in zip(L["p2p_tgt"], L["p2p_src"]):
        cnt[bb[t]:be[t], bb[s]:be[s]] += 1
    for t, s in zip(L["m2l_tgt"], L["m2l_src"]):
        cnt[bb[t]:be[t], bb[s]:be[s]] += 1
    assert np.all(cnt == 1)
    _, perm = T.keys()
    u = (np.asarray(x, np.float64)[perm, :3] - r["corner"]) * (2.0 ** 21 / r["H"])  # units of H / 2^21
    lev = c["level"].astype(np.int64)
    ijk = np.stack([c["ix"], c["iy"], c["iz"]], 1).astype(np.int64)
    ctr = ((2 * ijk + 1) << (21 - lev)[:, None]).astype(np.float64)
    rad = np.array([np.sqrt(((u[bb[i]:be[i]] - ctr[i]) ** 2).sum(1).max()) for i in range(lev.size)])
    assert np.all(rad <= np.sqrt(3.0) * np.ldexp(1.0, 21 - lev) + 1e-9)  # inside the cube
    slack = 2.0 * np.sqrt(3.0)  # a body sits at most one unit per axis from its voxel centre
    for t, s in zip(L["m2l_tgt"], L["m2l_src"]):
        d = np.sqrt(((ctr[t] - ctr[s]) ** 2).sum())
        assert theta * d > rad[t] + rad[s] - slack
    # the bound is tighter than the circumscribed sphere: fewer body pairs go to P2P
    C = orc.OracleTree(x, 4, theta, 8, circumscribed=True)
    assert T.info()["p2p_pairs"] < C.info()["p2p_pairs"]


def test_tight_mac_error_decreases_with_p(orc):
    x = W.plummer(3000, 53)
    pd, _ = orc.direct(x)
    e = [rel(orc.OracleTree(x, p, 0.5, 16, tight=True).evaluate()[0], pd) for p in (3, 5, 7, 9)]
    assert all(b < a for a, b in zip(e, e[1:]))


# ------------------------------------------- particle-fitted centres (f3)
# Sec. II.B: cells are squeezed to fit their particles.  With fitted=True the
# oracle takes every expansion about the centre of the box of the cell's
# bodies (their voxel centres 2u + 1, u the 21-bit coordinates; units of
# H / 2^21), and the MAC radius is the distance from there to the farthest
# voxel centre.  The pins below derive centres and radii here, from the
# bodies' coordinates, and check the oracle against them.

def _voxels(T):
    """(N, 3) int64 voxel coordinates u of the sorted bodies, from the keys
    (the keys themselves are pinned against their definition)."""
    keys, _ = T.keys()
    return np.stack([_deinterleave(keys, 2), _deinterleave(keys, 1), _deinterleave(keys, 0)], 1)


def _fitted_geometry(T):
    """Per cell: the integer centre u_min + u_max + 1 of its voxel box, the
    squared distance to its farthest voxel centre (exact integers) and the
    physical centre corner + centre * H / 2^21."""
    u = _voxels(T)
    c = T.cells()
    bb, be = c["body_begin"], c["body_end"]
    n = c["level"].size
    ctr = np.zeros((n, 3), np.int64)
    r2 = np.zeros(n, np.int64)
    for i in range(n):
        ui = u[bb[i]:be[i]]
        ctr[i] = ui.min(0) + ui.max(0) + 1
        r2[i] = int(((2 * ui + 1 - ctr[i]) ** 2).sum(1).max())
    r = T.root()
    phys = r["corner"][None, :] + ctr.astype(np.float64) * np.ldexp(r["H"], -21)
    return ctr, r2, phys


def test_fitted_centres_are_the_box_centres(orc):
    x = W.plummer(2500, 61)
    T = orc.OracleTree(x, 4, 0.5, 10, fitted=True)
    ctr, r2, phys = _fitted_geometry(T)
    assert np.array_equal(T.centres(), phys)
    # every body lies within the fitted radius of its cell's centre (up to
    # its voxel: one unit per axis)
    c = T.cells()
    bb, be = c["body_begin"], c["body_end"]
    _, perm = T.keys()
    r = T.root()
    xs = (np.asarray(x, np.float64)[perm, :3] - r["corner"]) * (2.0 ** 21 / r["H"])
    for i in range(ctr.shape[0]):
        d = np.sqrt(((xs[bb[i]:be[i]] - ctr[i]) ** 2).sum(1)).max()
        assert d <= math.sqrt(r2[i]) + math.sqrt(3.0) + 1e-6
    # a fitted box is never wider than its cube: the centre stays inside it
    lev = c["level"].astype(np.int64)
    ijk = np.stack([c["ix"], c["iy"], c["iz"]], 1).astype(np.int64)
    lo = (2 * ijk) << (21 - lev)[:, None]
    hi = (2 * ijk + 2) << (21 - lev)[:, None]
    assert np.all((ctr >= lo) & (ctr <= hi))


@pytest.mark.parametrize("theta", [0.5, 0.6])
def test_fitted_lists_follow_the_acceptance_criterion(orc, theta):
    """Every M2L pair passes theta |c_A - c_B| > r_A + r_B with the fitted
    centres and radii derived here, every P2P pair of distinct leaves fails
    it, and every body pair is covered exactly once."""
    x = W.plummer(1500, 62)
    T = orc.OracleTree(x, 4, theta, 8, fitted=True)
    ctr, r2, _ = _fitted_geometry(T)
    rad = [math.sqrt(float(v)) for v in r2]
    L = T.lists()

    def accepted(a, b):
        d = ctr[a] - ctr[b]
        s = rad[a] + rad[b]
        return (theta * theta) * float(int(d @ d)) > s * s

    assert len(L["m2l_tgt"]) > 0
    assert all(accepted(t, s) for t, s in zip(L["m2l_tgt"], L["m2l_src"]))
    far_p2p = [(t, s) for t, s in zip(L["p2p_tgt"], L["p2p_src"]) if t != s]
    assert not any(accepted(t, s) for t, s in far_p2p)
    c = T.cells()
    N = x.shape[0]
    bb, be = c["body_begin"], c["body_end"]
    cnt = np.zeros((N, N), np.int32)
    for key in (("p2p_tgt", "p2p_src"), ("m2l_tgt", "m2l_src")):
        for t, s in zip(L[key[0]], L[key[1]]):
            cnt[bb[t]:be[t], bb[s]:be[s]] += 1
    assert np.all(cnt == 1)
    # fitting the centres as well as the radii sends fewer body pairs to P2P
    Ttight = orc.OracleTree(x, 4, theta, 8, tight=True)
    assert T.info()["p2p_pairs"] < Ttight.info()["p2p_pairs"]


@pytest.mark.parametrize("dist,p", [("plummer", 4), ("cube", 5)])
def test_fitted_matches_cartesian_taylor_checker(orc, dist, p):
    """With the centres derived here, the basis-free double Taylor closed form
    equals the oracle: pins P2M/M2M/M2L/L2L/L2P about moved centres."""
    x = W.cube(600, 63) if dist == "cube" else W.plummer(600, 64)
    T = orc.OracleTree(x, p, 0.5, 12, fitted=True)
    assert T.info()["n_m2l"] > 0
    _, _, phys = _fitted_geometry(T)
    ph, g = T.evaluate()
    ph2, g2 = taylor_checker.evaluate(x, p, T.cells(), T.lists(), T.keys(), T.root(), centres=phys)
    assert rel(ph, ph2) < 1e-12
    assert rel(g, g2) < 1e-11


def test_fitted_error_decreases_with_p(orc):
    x = W.plummer(3000, 65)
    pd, _ = orc.direct(x)
    e = [rel(orc.OracleTree(x, p, 0.5, 16, fitted=True).evaluate()[0], pd) for p in (3, 5, 7, 9)]
    assert all(b < a for a, b in zip(e, e[1:]))


def test_fitted_operator_symmetry_and_adjoint(orc):
    """The double truncation about two moved centres is still symmetric
    (1/r is even), so w.FMM(q) = q.FMM(w) and the frozen-centre adjoint is the
    exact derivative: central differences (h = 1e-6) with the tree, lists and
    centres frozen agree with it."""
    rng = np.random.default_rng(66)
    N = 1024
    xyzq = np.concatenate([rng.random((N, 3)), rng.uniform(-1, 1, (N, 1))], axis=1)
    w = rng.standard_normal(N)
    T = orc.OracleTree(xyzq, 7, 0.5, 32, fitted=True)
    q0 = xyzq[:, 3].copy()
    pq, _ = T.evaluate(q=q0)
    pw, _ = T.evaluate(q=w)
    assert abs(w @ pq - q0 @ pw) <= 1e-12 * np.abs(w) @ np.abs(pq)
    dq, dx = T.backward(w)
    xyz0 = xyzq[:, :3].copy()

    def loss(xyz):
        return w @ T.evaluate(q=q0, xyz=xyz)[0]

    h = 1e-6
    for i in rng.choice(N, 12, replace=False):
        for a in range(3):
            xp = xyz0.copy(); xp[i, a] += h
            xm = xyz0.copy(); xm[i, a] -= h
            fd = (loss(xp) - loss(xm)) / (2 * h)
            assert abs(fd - dx[i, a]) <= 1e-6 * (abs(dx[i, a]) + 1e-3 * np.abs(dx).max())
    assert rel(dq, pw) < 1e-14


def _deinterleave(keys, shift):
    u = np.zeros(keys.shape, np.int64)
    for b in range(21):
        u |= ((keys >> np.uint64(3 * b + shift)) & np.uint64(1)).astype(np.int64) << b
    return u


@pytest.mark.parametrize("theta", [0.5, 0.55])
@pytest.mark.parametrize("mode", ["half", "circumscribed", "tight"])
def test_lists_follow_the_acceptance_criterion(orc, mode, theta):
    """Sec. II.A/C: a pair of cells goes to M2L exactly when it is far enough
    for its sizes.  Every M2L pair passes theta |c_A - c_B| > R_A + R_B and every
    P2P pair of two distinct leaves fails it, with the radii derived here from
    the geometry (units of H / 2^21): the half side 2^(21-l); the distance from
    the centre to a corner of the cube (the circumscribed sphere); the distance
    to the farthest voxel centre 2u + 1 of the cell's bodies (particle-fitted).
    At theta = 0.5 with the half side, cells two widths apart along an axis meet
    the criterion with equality; the strict inequality sends them to P2P."""
    x = W.plummer(2000, 54)
    T = orc.OracleTree(x, 4, theta, 6, circumscribed=mode == "circumscribed", tight=mode == "tight")
    c = T.cells()
    L = T.lists()
    lev = c["level"].astype(np.int64)
    ijk = np.stack([c["ix"], c["iy"], c["iz"]], 1).astype(np.int64)
    half = np.left_shift(np.int64(1), 21 - lev)
    ctr = (2 * ijk + 1) * half[:, None]
    if mode == "tight":
        keys, _ = T.keys()
        u = np.stack([_deinterleave(keys, 2), _deinterleave(keys, 1), _deinterleave(keys, 0)], 1)
        vox = 2 * u + 1
        bb, be = c["body_begin"], c["body_end"]
        r2 = np.array([int(((vox[bb[i]:be[i]] - ctr[i]) ** 2).sum(1).max()) for i in range(lev.size)])
        rad = [math.sqrt(float(v)) for v in r2]
    # a corner of the cube, (h, h, h) from its centre, is sqrt(3) h away
    k2 = 3 if mode == "circumscribed" else 1

    def accepted(a, b):
        d = ctr[a] - ctr[b]
        D2 = int(d @ d)
        if mode == "tight":
            s = rad[a] + rad[b]
            return (theta * theta) * float(D2) > s * s
        # (R_A + R_B)^2 = k^2 (h_A + h_B)^2, exact in integers
        return (theta * theta) * float(D2) > float(k2 * (int(half[a]) + int(half[b])) ** 2)

    assert len(L["m2l_tgt"]) > 0
    assert all(accepted(t, s) for t, s in zip(L["m2l_tgt"], L["m2l_src"]))
    far_p2p = [(t, s) for t, s in zip(L["p2p_tgt"], L["p2p_src"]) if t != s]
    assert len(far_p2p) > 0
    assert not any(accepted(t, s) for t, s in far_p2p)
    if mode == "half" and theta == 0.5:
        def tie(a, b):
            d = ctr[a] - ctr[b]
            return (theta * theta) * float(int(d @ d)) == float((int(half[a]) + int(half[b])) ** 2)
        assert any(tie(t, s) for t, s in far_p2p)


def test_coincident_bodies_contribute_zero(orc):
    x = W.cube(300, 61)
    x[10, :3] = x[20, :3]
    x[11, :3] = x[20, :3]
    T = orc.OracleTree(x, 5, 0.5, 8)
    ph, g = T.evaluate()
    pd, gd = orc.direct(x)
    assert np.all(np.isfinite(ph)) and rel(ph, pd) < 1e-3


def test_depth_capped_leaf(orc):
    """All bodies at one point: the tree stops at level 21 with an oversized leaf."""
    x = np.tile(np.array([[0.3, 0.3, 0.3, 1.0]], np.float32), (50, 1))
    T = orc.OracleTree(x, 4, 0.5, 4)
    c = T.cells()
    assert c["level"].max() == 21
    ph, g = T.evaluate()
    assert np.all(ph == 0) and np.all(g == 0)


# ----------------------------------------------------------- invariants

def test_linearity_in_charges(orc):
    x = W.cube(3000, 71)
    T = orc.OracleTree(x, 6, 0.4, 32)
    q1 = W.cube(3000, 72)[:, 3].astype(np.float64)
    q2 = W.cube(3000, 73)[:, 3].astype(np.float64)
    a1, g1 = T.evaluate(q=q1)
    a2, g2 = T.evaluate(q=q2)
    a3, g3 = T.evaluate(q=2.0 * q1 - 3.0 * q2)
    assert rel(a3, 2 * a1 - 3 * a2) < 1e-13 and rel(g3, 2 * g1 - 3 * g2) < 1e-13


def test_power_of_two_scaling(orc):
    """x -> 2x keeps the tree and gives phi/2, grad/4 exactly."""
    x = W.cube(2000, 81).astype(np.float64)
    T1 = orc.OracleTree(x, 6, 0.4, 32)
    y = x.copy(); y[:, :3] *= 2.0
    T2 = orc.OracleTree(y, 6, 0.4, 32)
    assert np.array_equal(T1.keys()[0], T2.keys()[0])
    a, g = T1.evaluate()
    b, h = T2.evaluate()
    assert np.array_equal(b * 2, a) and np.array_equal(h * 4, g)


def test_dyadic_translation(orc):
    x = W.cube(2000, 82).astype(np.float64)
    T1 = orc.OracleTree(x, 6, 0.4, 32)
    y = x.copy(); y[:, :3] += np.array([0.5, -1.0, 2.0])
    T2 = orc.OracleTree(y, 6, 0.4, 32)
    assert np.array_equal(T1.keys()[0], T2.keys()[0])
    a, g = T1.evaluate()
    b, h = T2.evaluate()
    assert rel(b, a) < 1e-12 and rel(h, g) < 1e-11


def test_axis_permutation_equivariance(orc):
    x = W.cube(2000, 83).astype(np.float64)
    a, g = orc.OracleTree(x, 7, 0.4, 32).evaluate()
    y = x[:, [1, 2, 0, 3]]
    b, h = orc.OracleTree(y, 7, 0.4, 32).evaluate()
    assert rel(b, a) < 1e-12 and rel(h, g[:, [1, 2, 0]]) < 1e-11


def test_newton_third_law(orc):
    x = W.cube(4096, 84)
    T = orc.OracleTree(x, 8, 0.4, 64)
    _, g = T.evaluate()
    q = x[:, 3].astype(np.float64)
    f = -q[:, None] * g
    pd, gd = orc.direct(x)
    err = rel(g, gd)
    assert np.linalg.norm(f.sum(0)) / np.abs(f).sum() < 10 * err


def test_operator_symmetry(orc):
    """w . FMM(q) == q . FMM(w): the lists and the double truncation are symmetric."""
    x = W.cube(3000, 85)
    T = orc.OracleTree(x, 6, 0.5, 24)
    q = x[:, 3].astype(np.float64)
    w = W.weights(3000, 86).astype(np.float64)
    pq, _ = T.evaluate(q=q)
    pw, _ = T.evaluate(q=w)
    assert abs(w @ pq - q @ pw) <= 1e-12 * np.abs(w) @ np.abs(pq)


# -------------------------------------------------------------- adjoint

def test_adjoint_matches_central_differences(orc):
    """Frozen tree, double precision, h = 1e-6: dL/dq and dL/dx of
    L = sum w_i phi_i agree with central differences."""
    rng = np.random.default_rng(41)
    N = 1024
    xyzq = np.concatenate([rng.random((N, 3)), rng.uniform(-1, 1, (N, 1))], axis=1)
    w = rng.standard_normal(N)
    T = orc.OracleTree(xyzq, 8, 0.4, 64)
    dq, dx = T.backward(w)
    xyz0 = xyzq[:, :3].copy()
    q0 = xyzq[:, 3].copy()

    def loss(xyz, q):
        return w @ T.evaluate(q=q, xyz=xyz)[0]

    h = 1e-6
    for i in rng.choice(N, 24, replace=False):
        for a in range(3):
            xp = xyz0.copy(); xp[i, a] += h
            xm = xyz0.copy(); xm[i, a] -= h
            fd = (loss(xp, q0) - loss(xm, q0)) / (2 * h)
            assert abs(fd - dx[i, a]) <= 1e-6 * (abs(dx[i, a]) + 1e-3 * np.abs(dx).max())
        qp = q0.copy(); qp[i] += h
        qm = q0.copy(); qm[i] -= h
        fd = (loss(xyz0, qp) - loss(xyz0, qm)) / (2 * h)
        # L is linear in q: the only error is the rounding of L over 2h
        assert abs(fd - dq[i]) <= 1e-6 * (abs(dq[i]) + 1)
        q1 = q0.copy(); q1[i] += 1.0
        assert abs((loss(xyz0, q1) - loss(xyz0, q0)) - dq[i]) <= 1e-10 * (abs(dq[i]) + 1)


def test_adjoint_vs_direct_gradient(orc):
    x = W.cube(4096, 4)
    w = W.weights(4096, 40).astype(np.float64)
    T = orc.OracleTree(x, 8, 0.4, 64)
    dq, dx = T.backward(w)
    q = x[:, 3].astype(np.float64)
    pw, gw = orc.direct(np.concatenate([x[:, :3].astype(np.float64), w[:, None]], 1))
    _, gq = orc.direct(x)
    # FMM truncation error at p = 8 is ~1e-5 (see test_error_decreases_with_p)
    assert rel(dq, pw) < 1e-4
    assert rel(dx, w[:, None] * gq + q[:, None] * gw) < 1e-4


# ---------------------------------------------------------------- paper

def test_table1_parameters_fixture():
    """The paper's Table 1 (printed): the Cube and Plummer cases use P = 10,
    theta = 0.4; the workloads keep those where they claim Table 1 shapes."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_parameters.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    tab = {r[6]: dict(N=float(r[1]), P=int(r[2]), theta=float(r[3]), ncrit=int(r[4])) for r in rows}
    assert tab["Cube"]["P"] == 10 and tab["Cube"]["theta"] == 0.4
    assert W.WORKLOADS["cube1m_p10"]["p"] == tab["Cube"]["P"]
    assert W.WORKLOADS["cube1m_p10"]["theta"] == tab["Cube"]["theta"]
    assert tab["Plummer"]["ncrit"] == 64 and tab["Sphere"]["ncrit"] == 512
