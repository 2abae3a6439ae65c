"""Parity of the CUDA path (through the C ABI) with the double-precision oracle.

Integer and index work (keys, permutation, cells, interaction lists) must be
bit-identical.  Floating point: single precision must match the oracle to a
relative L2 error of 1e-5 (potential) and 1e-4 (force) at equal p, theta and
ncrit; double precision to 1e-11 / 1e-10.
"""

import numpy as np
import pytest
import torch

from paper_1405_7487_gb300 import workloads as W
from tests.gpu_helpers import assert_match, rel, scale_oracle, unpack

pytestmark = pytest.mark.gpu

TOL_PHI, TOL_F = 1e-5, 1e-4
TOL64_PHI, TOL64_F = 1e-11, 1e-10


@pytest.fixture(scope="module")
def fmm():
    from paper_1405_7487_gb300 import build_lib
    build_lib.build()
    from paper_1405_7487_gb300 import fmm as F
    assert torch.cuda.is_available()
    return F


def gpu_tree(F, x, p, theta, ncrit, flags=0, f64=False):
    t = torch.from_numpy(np.asarray(x, np.float64 if f64 else np.float32)).cuda()
    return F.Tree(t, p, theta, ncrit, flags)


def evaluate(tree):
    pot, force = tree.evaluate()
    torch.cuda.synchronize()
    return pot.double().cpu().numpy(), force.double().cpu().numpy()


CASES = {
    "cube4k_p4": (lambda: W.cube(4096, 1), 4, 0.4, 64),
    "cube65k_p10": (lambda: W.cube(65536, 12), 10, 0.4, 64),
    "plummer60k_p8": (lambda: W.plummer(60000, 13), 8, 0.5, 32),
    "sphere40k_p6": (lambda: W.sphere(40000, 14), 6, 0.4, 64),
    "cube20k_p16": (lambda: W.cube(20000, 15), 16, 0.4, 32),
    "cube3k_p1": (lambda: W.cube(3000, 16), 1, 0.5, 8),
}


# ------------------------------------------------------------ structure

@pytest.mark.parametrize("name", ["cube4k_p4", "plummer60k_p8", "sphere40k_p6"])
@pytest.mark.parametrize("mac", ["half", "circ", "tight", "fitted"])
def test_tree_and_lists_bit_identical(fmm, orc, name, mac):
    gen, p, theta, ncrit = CASES[name]
    x = gen()
    flags = {"half": 0, "circ": fmm.FMM_FLAG_CIRCUMSCRIBED, "tight": fmm.FMM_FLAG_TIGHT_MAC,
             "fitted": fmm.FMM_FLAG_FITTED_CENTRES}[mac]
    T = gpu_tree(fmm, x, p, theta, ncrit, flags)
    O = orc.OracleTree(x, p, theta, ncrit, circumscribed=mac == "circ", tight=mac == "tight",
                       fitted=mac == "fitted")
    r_g, r_o = T.root(), O.root()
    for k in ("lo", "hi", "centre", "corner"):
        assert np.array_equal(r_g[k], r_o[k])
    assert r_g["H"] == r_o["H"]
    kg, pg = T.keys()
    ko, po = O.keys()
    assert np.array_equal(kg, ko)
    assert np.array_equal(pg.astype(np.int64), po)
    cg, co = T.cells(), O.cells()
    for k in co:
        assert np.array_equal(cg[k], co[k]), k
    lg, lo = T.lists(), O.lists()
    for k in lo:
        assert np.array_equal(lg[k], lo[k]), k
    st = T.stats()
    assert st["n_p2p_body_pairs"] == O.info()["p2p_pairs"]


def test_coincident_and_capped_tree_identical(fmm, orc):
    x = W.cube(2000, 17)
    x[100:160, :3] = x[5, :3]  # 61 bodies at one point: a level-21 leaf
    T = gpu_tree(fmm, x, 5, 0.5, 16)
    O = orc.OracleTree(x, 5, 0.5, 16)
    assert np.array_equal(T.keys()[0], O.keys()[0])
    for k, v in O.cells().items():
        assert np.array_equal(T.cells()[k], v)
    assert T.cells()["level"].max() == 21
    ph, f = evaluate(T)
    po, go = O.evaluate()
    assert np.all(np.isfinite(ph)) and rel(ph, po) < TOL_PHI and rel(f, -go) < TOL_F


# ---------------------------------------------------------- expansions

def test_expansions_match_oracle(fmm, orc):
    x = W.cube(30000, 18)
    p = 8
    T = gpu_tree(fmm, x, p, 0.4, 32)
    O = orc.OracleTree(x, p, 0.4, 32)
    evaluate(T)
    O.evaluate()
    Mg, Lg = T.expansions()
    Mo, Lo = O.expansions()
    cells = O.cells()
    R = np.ldexp(O.root()["H"], -cells["level"].astype(np.int64))
    Ms, Ls = scale_oracle(Mo, Lo, R, p)
    assert rel(unpack(Mg.astype(np.float64), p), Ms) < 1e-6
    assert rel(unpack(Lg.astype(np.float64), p), Ls) < 1e-5


# -------------------------------------------------------------- outputs

@pytest.mark.parametrize("name", list(CASES))
def test_forward_matches_oracle(fmm, orc, name):
    gen, p, theta, ncrit = CASES[name]
    x = gen()
    T = gpu_tree(fmm, x, p, theta, ncrit)
    ph, f = evaluate(T)
    po, go = orc.OracleTree(x, p, theta, ncrit).evaluate()
    assert_match(ph, po, f, -go, TOL_PHI, TOL_F)


@pytest.mark.parametrize("name,f64", [("cube65k_p10", False), ("plummer60k_p8", False), ("sphere40k_p6", False),
                                      ("cube4k_p4", True)])
def test_tight_mac_matches_oracle(fmm, orc, name, f64):
    """Particle-fitted MAC radius (row f3, centres kept): outputs against the
    oracle built with the same MAC, forward and backward."""
    gen, p, theta, ncrit = CASES[name]
    x = gen()
    T = gpu_tree(fmm, x, p, theta, ncrit, fmm.FMM_FLAG_TIGHT_MAC, f64=f64)
    ph, f = evaluate(T)
    O = orc.OracleTree(x, p, theta, ncrit, tight=True)
    po, go = O.evaluate()
    tp, tf = (TOL64_PHI, TOL64_F) if f64 else (TOL_PHI, TOL_F)
    assert rel(ph, po) < tp and rel(f, -go) < tf
    w = W.weights(x.shape[0], 31)
    dq, dx = T.backward(torch.from_numpy(np.asarray(w, np.float64 if f64 else np.float32)).cuda())
    torch.cuda.synchronize()
    dqo, dxo = O.backward(np.asarray(w, np.float64))
    assert rel(dq.double().cpu().numpy(), dqo) < tp and rel(dx.double().cpu().numpy(), dxo) < tf


@pytest.mark.parametrize("name,f64", [("cube65k_p10", False), ("plummer60k_p8", False), ("sphere40k_p6", False),
                                      ("cube20k_p16", False), ("cube3k_p1", False), ("cube4k_p4", True),
                                      ("plummer60k_p8", True)])
def test_fitted_centres_match_oracle(fmm, orc, name, f64):
    """Expansion centres at the particle-fitted boxes (row f3): M2M, L2L and M2L
    per pair about the moved centres, against the oracle built the same way,
    forward and backward (frozen centres), single and double precision."""
    gen, p, theta, ncrit = CASES[name]
    x = gen()
    T = gpu_tree(fmm, x, p, theta, ncrit, fmm.FMM_FLAG_FITTED_CENTRES, f64=f64)
    assert T.stats()["m2l_engine"] == 3
    ph, f = evaluate(T)
    O = orc.OracleTree(x, p, theta, ncrit, fitted=True)
    po, go = O.evaluate()
    tp, tf = (TOL64_PHI, TOL64_F) if f64 else (TOL_PHI, TOL_F)
    bp, bf = (1e-9, 1e-8) if f64 else (1e-4, 1e-3)
    assert_match(ph, po, f, -go, tp, tf, bp, bf)
    Mg, Lg = T.expansions()
    Mo, Lo = O.expansions()
    cells = O.cells()
    R = np.ldexp(O.root()["H"], -cells["level"].astype(np.int64))
    Ms, Ls = scale_oracle(Mo, Lo, R, p)
    assert rel(unpack(Mg.astype(np.float64), p), Ms) < (1e-12 if f64 else 1e-6)
    assert rel(unpack(Lg.astype(np.float64), p), Ls) < (1e-11 if f64 else 1e-5)
    w = W.weights(x.shape[0], 32)
    dq, dx = T.backward(torch.from_numpy(np.asarray(w, np.float64 if f64 else np.float32)).cuda())
    torch.cuda.synchronize()
    dqo, dxo = O.backward(np.asarray(w, np.float64))
    assert_match(dq.double().cpu().numpy(), dqo, dx.double().cpu().numpy(), dxo, tp, tf, bp, bf)
    T.check()


@pytest.mark.parametrize("name,f64", [("cube65k_p10", False), ("plummer60k_p8", False), ("sphere40k_p6", False),
                                      ("cube4k_p4", True)])
def test_mutual_p2p_matches_oracle(fmm, orc, name, f64):
    """Mutual interaction (each unordered leaf pair once, both sides updated
    through atomics) gives the oracle's result, forward and backward."""
    gen, p, theta, ncrit = CASES[name]
    x = gen()
    T = gpu_tree(fmm, x, p, theta, ncrit, fmm.FMM_FLAG_MUTUAL_P2P, f64=f64)
    ph, f = evaluate(T)
    O = orc.OracleTree(x, p, theta, ncrit)
    po, go = O.evaluate()
    tp, tf = (1e-11, 1e-10) if f64 else (TOL_PHI, TOL_F)
    assert rel(ph, po) < tp
    assert rel(f, -go) < tf
    w = W.weights(x.shape[0], 31)
    wt = torch.from_numpy(w.astype(np.float64 if f64 else np.float32)).cuda()
    dq, dx = T.backward(wt)
    torch.cuda.synchronize()
    dqo, dxo = O.backward(w.astype(np.float64))
    assert rel(dq.double().cpu().numpy(), dqo) < tp
    assert rel(dx.double().cpu().numpy(), dxo) < tf


def test_charges_override_and_repeat(fmm, orc):
    x = W.cube(20000, 19)
    q2 = W.weights(20000, 20)
    T = gpu_tree(fmm, x, 6, 0.4, 64)
    a1, f1 = evaluate(T)
    pot2, force2 = T.evaluate(torch.from_numpy(q2).cuda())
    a3, f3 = evaluate(T)
    assert np.array_equal(a1, a3) and np.array_equal(f1, f3)  # deterministic, build charges restored
    O = orc.OracleTree(x, 6, 0.4, 64)
    po, go = O.evaluate(q=q2.astype(np.float64))
    assert rel(pot2.double().cpu().numpy(), po) < TOL_PHI
    assert rel(force2.double().cpu().numpy(), -go) < TOL_F


def test_force_optional(fmm):
    x = torch.from_numpy(W.cube(5000, 21)).cuda()
    T = fmm.Tree(x, 4, 0.4, 64)
    pot, force = T.evaluate(force=False)
    assert force is None
    pot2, _ = T.evaluate()
    assert torch.equal(pot, pot2)


@pytest.mark.parametrize("wl", ["cube1m_p10", "plummer1m_p8", "sphere1m_p10"])
def test_full_size_sampled_parity(fmm, orc, wl):
    """The benchmark workloads at full size: 4096 sampled targets against the
    oracle (same tree) and the error against the double direct sum."""
    spec = W.WORKLOADS[wl]
    x = W.make(wl)
    T = gpu_tree(fmm, x, spec["p"], spec["theta"], spec["ncrit"])
    ph, f = evaluate(T)
    idx = W.sample_targets(x.shape[0], 4096)
    O = orc.OracleTree(x, spec["p"], spec["theta"], spec["ncrit"])
    po, go = O.evaluate(targets=idx)
    assert_match(ph[idx], po, f[idx], -go, TOL_PHI, TOL_F)
    pd, gd = orc.direct(x, targets=idx)
    err_phi, err_f = rel(ph[idx], pd), rel(f[idx], -gd)
    eo_phi = rel(po, pd)
    assert err_phi < max(2 * eo_phi, 1e-5), (err_phi, eo_phi)
    assert err_f < 1e-3


# ---------------------------------------------------------------- adjoint

def test_backward_matches_oracle(fmm, orc):
    x = W.cube(40000, 22)
    w = W.weights(40000, 23)
    T = gpu_tree(fmm, x, 8, 0.4, 64)
    evaluate(T)
    dq, dx = T.backward(torch.from_numpy(w).cuda())
    torch.cuda.synchronize()
    O = orc.OracleTree(x, 8, 0.4, 64)
    dqo, dxo = O.backward(w.astype(np.float64))
    assert_match(dq.double().cpu().numpy(), dqo, dx.double().cpu().numpy(), dxo, TOL_PHI, TOL_F)


def test_backward_before_evaluate_is_state_error(fmm):
    x = torch.from_numpy(W.cube(3000, 24)).cuda()
    T = fmm.Tree(x, 4, 0.4, 64)
    with pytest.raises(fmm.FMMError) as e:
        T.backward(torch.ones(3000, device="cuda"))
    assert e.value.name == "FMM_ERR_STATE"


def test_autograd_function(fmm, orc):
    x0 = W.cube(262144, 4)
    w = W.weights(262144, 40)
    x = torch.from_numpy(x0[:, :3]).cuda().requires_grad_(True)
    q = torch.from_numpy(x0[:, 3]).cuda().requires_grad_(True)
    wt = torch.from_numpy(w).cuda()
    phi, force = fmm.FMM(8, 0.4, 64)(x, q)
    (phi * wt).sum().backward()
    O = orc.OracleTree(x0, 8, 0.4, 64)
    idx = W.sample_targets(262144, 4096)
    dqo, dxo = O.backward(w.astype(np.float64))
    assert rel(q.grad.double().cpu().numpy(), dqo) < TOL_PHI
    assert rel(x.grad.double().cpu().numpy(), dxo) < TOL_F
    # against the direct-sum gradient on sampled bodies (FMM error level)
    xyzq = x0.astype(np.float64)
    _, gq = orc.direct(xyzq, targets=idx)
    pw, gw = orc.direct(np.concatenate([xyzq[:, :3], w[:, None].astype(np.float64)], 1), targets=idx)
    dx_direct = w[idx, None] * gq + xyzq[idx, 3:4] * gw
    assert rel(q.grad.double().cpu().numpy()[idx], pw) < 1e-4
    assert rel(x.grad.double().cpu().numpy()[idx], dx_direct) < 1e-3


# ---------------------------------------------------------- double path

@pytest.mark.parametrize("name", ["cube4k_p4", "plummer60k_p8"])
def test_double_precision_path(fmm, orc, name):
    gen, p, theta, ncrit = CASES[name]
    x = gen().astype(np.float64)
    T = gpu_tree(fmm, x, p, theta, ncrit, f64=True)
    ph, f = evaluate(T)
    O = orc.OracleTree(x, p, theta, ncrit)
    po, go = O.evaluate()
    assert_match(ph, po, f, -go, TOL64_PHI, TOL64_F, 1e-9, 1e-8)
    w = W.weights(x.shape[0], 25).astype(np.float64)
    dq, dx = T.backward(torch.from_numpy(w).cuda())
    dqo, dxo = O.backward(w)
    assert_match(dq.cpu().numpy(), dqo, dx.cpu().numpy(), dxo, TOL64_PHI, TOL64_F, 1e-9, 1e-8)


# ------------------------------------------------------------ edge cases

def test_single_body_and_pairs(fmm, orc):
    one = np.array([[0.3, 0.2, 0.1, 1.0]], np.float32)
    T = gpu_tree(fmm, one, 4, 0.4, 64)
    ph, f = evaluate(T)
    assert ph[0] == 0.0 and np.all(f == 0.0)
    two = np.array([[0.0, 0.0, 0.0, 1.0], [1.0, 0.0, 0.0, 2.0]], np.float32)
    ph, f = evaluate(gpu_tree(fmm, two, 4, 0.4, 1))
    assert np.allclose(ph, [2.0, 1.0]) and np.allclose(f[:, 0], [-2.0, 1.0])


def test_root_leaf_equals_direct(fmm, orc):
    x = W.cube(3000, 26)
    ph, f = evaluate(gpu_tree(fmm, x, 6, 0.4, 5000))
    pd, gd = orc.direct(x)
    assert rel(ph, pd) < 1e-6 and rel(f, -gd) < 1e-5


def test_all_coincident(fmm):
    x = np.tile(np.array([[0.5, 0.5, 0.5, 1.0]], np.float32), (300, 1))
    ph, f = evaluate(gpu_tree(fmm, x, 4, 0.4, 8))
    assert np.all(ph == 0) and np.all(f == 0)


def test_ragged_tiles_and_deep_tree(fmm, orc):
    """ncrit = 1 gives a deep tree and tiles/ranges with ragged tails."""
    x = W.plummer(5000, 27)
    ph, f = evaluate(gpu_tree(fmm, x, 5, 0.5, 1))
    po, go = orc.OracleTree(x, 5, 0.5, 1).evaluate()
    assert rel(ph, po) < TOL_PHI and rel(f, -go) < TOL_F


@pytest.mark.parametrize("n, ncrit", [(4099, 7), (1201, 600), (2047, 300)])
def test_odd_sizes_and_multi_chunk_leaves(fmm, orc, n, ncrit):
    """Odd body counts (the last source pair has one body) and leaves of more
    than 256 bodies (several near-field work items per leaf, one of them
    ragged)."""
    x = W.plummer(n, 29) if ncrit < 64 else W.cube(n, 29)
    ph, f = evaluate(gpu_tree(fmm, x, 6, 0.5, ncrit))
    po, go = orc.OracleTree(x, 6, 0.5, ncrit).evaluate()
    assert rel(ph, po) < TOL_PHI and rel(f, -go) < TOL_F


def test_long_neighbour_lists(fmm, orc):
    """theta = 0.1 and one body per leaf: about 1,000 target leaves with more
    than 1,024 source leaves (the long-list path of the per-leaf source sort)
    and 345 with more than 256 merged ranges (several staged range windows in
    the single-precision near field)."""
    x = W.cube(4000, 33)
    T = gpu_tree(fmm, x, 2, 0.1, 1)
    O = orc.OracleTree(x, 2, 0.1, 1)
    lg, lo = T.lists(), O.lists()
    for k in lo:
        assert np.array_equal(lg[k], lo[k]), k
    P = T.plan()
    rp, rg = P["p2p_rptr"], P["p2p_ranges"]
    assert np.diff(rp).max() > 256
    for li in range(rp.shape[0] - 1):
        r = rg[rp[li]:rp[li + 1]]
        assert np.all(r[1:, 0] > r[:-1, 1])  # ascending, disjoint and merged
    ph, f = evaluate(T)
    po, go = O.evaluate()
    assert rel(ph, po) < TOL_PHI and rel(f, -go) < TOL_F


def test_argument_errors(fmm):
    L = fmm.lib()
    x = torch.from_numpy(W.cube(100, 28)).cuda()
    import ctypes
    h = ctypes.c_void_p()
    ptr = ctypes.c_void_p(x.data_ptr())
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    bad = [(None, 100, 4, 0.4, 8), (ptr, 0, 4, 0.4, 8), (ptr, 100, 0, 0.4, 8), (ptr, 100, 17, 0.4, 8),
           (ptr, 100, 4, 0.0, 8), (ptr, 100, 4, 1.0, 8), (ptr, 100, 4, float("nan"), 8), (ptr, 100, 4, 0.4, 0)]
    for a in bad:
        assert L.fmm_build(a[0], a[1], a[2], a[3], a[4], 0, None, s, ctypes.byref(h)) == -1
        assert h.value is None
    xn = x.clone()
    xn[7, 1] = float("nan")
    assert L.fmm_build(ctypes.c_void_p(xn.data_ptr()), 100, 4, 0.4, 8, 0, None, s, ctypes.byref(h)) == -2
    T = fmm.Tree(x, 4, 0.4, 8)
    pot = torch.empty(100, dtype=torch.float64, device="cuda")
    assert L.fmm_evaluate_f64(T.handle, None, ctypes.c_void_p(pot.data_ptr()), None, s) == -6
    assert L.fmm_evaluate(T.handle, None, None, None, s) == -1
    assert L.fmm_destroy(None) == 0


def test_solve_host_equals_device_path(fmm):
    x = W.cube(50000, 29)
    w = W.weights(50000, 30)
    out = fmm.solve_host(x, w, 8, 0.4, 64)
    T = gpu_tree(fmm, x, 8, 0.4, 64)
    pot, force = T.evaluate()
    dq, dx = T.backward(torch.from_numpy(w).cuda())
    assert np.array_equal(out["pot"], pot.cpu().numpy())
    assert np.array_equal(out["force"], force.cpu().numpy())
    assert np.array_equal(out["dq"], dq.cpu().numpy())
    assert np.array_equal(out["dx"], dx.cpu().numpy())


def test_build_is_deterministic(fmm):
    x = W.plummer(100000, 31)
    a = evaluate(gpu_tree(fmm, x, 8, 0.5, 32))
    b = evaluate(gpu_tree(fmm, x, 8, 0.5, 32))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


# ----------------------------------------------------------- work plans

@pytest.mark.parametrize("name", ["cube4k_p4", "plummer60k_p8", "cube3k_p1"])
@pytest.mark.parametrize("f64", [False, True])
def test_plan_in_bounds_and_covers_lists(fmm, name, f64):
    """Every index of the M2L tiles/entries and of the P2P source ranges is in
    range, the (target, source) pairs of the M2L plan are exactly the M2L list,
    and the P2P ranges plus the leaf itself are exactly the P2P list's bodies."""
    gen, p, theta, ncrit = CASES[name]
    T = gpu_tree(fmm, gen(), p, theta, ncrit, f64=f64)
    st = T.stats()
    P = T.plan()
    L = T.lists()
    C = T.cells()
    nc, N = st["n_cells"], st["n_bodies"]
    tt, es = P["tile_tgt"], P["entry_src"]
    assert np.all((tt >= -1) & (tt < nc)) and np.all((es >= -1) & (es < nc))
    assert np.all((P["entry_class"] >= 0) & (P["entry_class"] < st["n_m2l_classes"]))
    ep = P["tile_eptr"]
    assert ep[0] == 0 and ep[-1] == es.shape[0] and np.all(np.diff(ep) >= 0)
    pairs = set()
    for t in range(tt.shape[0]):
        for e in range(ep[t], ep[t + 1]):
            for slot in np.nonzero(es[e] >= 0)[0]:
                assert tt[t, slot] >= 0
                pairs.add((int(tt[t, slot]), int(es[e, slot])))
    assert len(pairs) == st["n_m2l"]
    assert pairs == set(zip(L["m2l_tgt"].tolist(), L["m2l_src"].tolist()))
    rp, rg = P["p2p_rptr"], P["p2p_ranges"]
    assert rp[0] == 0 and rp[-1] == rg.shape[0] and np.all(np.diff(rp) >= 0)
    assert np.all((rg[:, 0] >= 0) & (rg[:, 1] <= N) & (rg[:, 0] < rg[:, 1]))
    leaves = np.nonzero(C["child_count"] == 0)[0]
    bb, be = C["body_begin"], C["body_end"]
    want = {}
    for t, s in zip(L["p2p_tgt"], L["p2p_src"]):
        want.setdefault(int(t), []).append((int(bb[s]), int(be[s])))
    for li, cell in enumerate(leaves):
        got = [(int(bb[cell]), int(be[cell]))] + [tuple(map(int, r)) for r in rg[rp[li]:rp[li + 1]]]
        cover = np.zeros(N, np.int32)
        for a, b in got:
            cover[a:b] += 1
        ref = np.zeros(N, np.int32)
        for a, b in want[int(cell)]:
            ref[a:b] += 1
        assert np.array_equal(cover, ref)


@pytest.mark.parametrize("name", ["cube65k_p10", "plummer60k_p8", "sphere40k_p6", "cube3k_p1"])
def test_dense_and_sorted_plans_identical(fmm, name):
    """The M2L plan numbered through dense key tables equals the plan numbered
    by sorting the pairs, array for array, and so do the outputs."""
    gen, p, theta, ncrit = CASES[name]
    x = gen()
    A = gpu_tree(fmm, x, p, theta, ncrit)
    B = gpu_tree(fmm, x, p, theta, ncrit, fmm.FMM_FLAG_SORTED_PLAN)
    assert A.stats()["n_m2l_classes"] == B.stats()["n_m2l_classes"]
    PA, PB = A.plan(), B.plan()
    assert PA.keys() == PB.keys()
    for k in PA:
        assert np.array_equal(PA[k], PB[k]), k
    pa, fa = evaluate(A)
    pb, fb = evaluate(B)
    assert np.array_equal(pa, pb) and np.array_equal(fa, fb)


@pytest.mark.parametrize("name", ["cube4k_p4", "cube65k_p10", "cube20k_p16", "cube3k_p1", "sphere40k_p6"])
def test_m2l_engines_agree(fmm, name):
    """The tensor-core M2L (3xTF32, tcgen05) and the CUDA-core M2L give the same
    local expansions to single-precision accuracy."""
    gen, p, theta, ncrit = CASES[name]
    x = gen()
    A = gpu_tree(fmm, x, p, theta, ncrit)
    B = gpu_tree(fmm, x, p, theta, ncrit, fmm.FMM_FLAG_M2L_CUDA_CORE)
    assert A.stats()["m2l_engine"] in (1, 2) and B.stats()["m2l_engine"] == 0
    pa, fa = evaluate(A)
    pb, fb = evaluate(B)
    La = A.expansions()[1].astype(np.float64)
    Lb = B.expansions()[1].astype(np.float64)
    # 3xTF32 products with TF32-rounded halves and chunked fp32 accumulation
    # differ from plain fp32 by a few 1e-6 (both are checked against the
    # oracle by the other tests)
    assert rel(La, Lb) < 3e-5
    assert rel(pa, pb) < 1e-5 and rel(fa, fb) < 5e-5
    assert A.stats()["device_errors"] == 0


@pytest.mark.parametrize("flags_name", ["default", "fitted"])
def test_fallback_build_paths_identical(fmm, flags_name):
    """The tree build and the traversal each run as one cooperative launch
    into buffers sized ahead; when a tree outgrows them, the tree build
    repeats at its bound and the traversal hands over to per-level launches.
    Forcing both (tiny first buffers through GBFMM_TREE_CELLS and
    GBFMM_TRAVERSE_BUDGET) must give the same cells, lists and outputs bit
    for bit, with more host synchronisations."""
    import os
    flags = 0 if flags_name == "default" else fmm.FMM_FLAG_FITTED_CENTRES
    x_h = W.plummer(60000, 61)
    x = torch.from_numpy(x_h).cuda()

    def run():
        T = fmm.Tree(x, 8, 0.5, 32, flags)
        pot, force = T.evaluate()
        torch.cuda.synchronize()
        out = (T.cells(), T.lists(), pot.cpu().numpy(), force.cpu().numpy(), T.stats())
        T.close()
        return out

    c0, l0, p0, f0, s0 = run()
    os.environ["GBFMM_TREE_CELLS"] = "64"
    os.environ["GBFMM_TRAVERSE_BUDGET"] = "1000"
    try:
        c1, l1, p1, f1, s1 = run()
    finally:
        del os.environ["GBFMM_TREE_CELLS"]
        del os.environ["GBFMM_TRAVERSE_BUDGET"]
    for k in c0:
        assert np.array_equal(c0[k], c1[k]), k
    for k in l0:
        assert np.array_equal(l0[k], l1[k]), k
    assert np.array_equal(p0, p1) and np.array_equal(f0, f1)
    assert s1["build_host_syncs"] > s0["build_host_syncs"]
    assert s0["device_errors"] == 0 and s1["device_errors"] == 0
