"""Parity at the benchmark's own sizes, through the C ABI.

* The headline workload (cube1m_p10: 1,048,576 bodies, p = 10, theta = 0.4,
  ncrit = 64) compared with the oracle on every body, forward (potential,
  force) and backward (dL/dq, dL/dx of sum w_i phi_i), with the relative L2
  tolerances and a per-body bound.
* The precision and scale sweep's workload (cube16m: 16,777,216 bodies,
  Table 1 / Sec. III scale) at p = 8 (four tiles per tensor-core block),
  p = 16 (one tile per block, 256 padded coefficients) in single precision
  and p = 4 in double precision, on sampled targets.  One oracle tree serves
  the three orders (the lists do not depend on p).
"""

import numpy as np
import pytest
import torch

from paper_1405_7487_gb300 import workloads as W
from tests.gpu_helpers import assert_match

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


def test_headline_whole_n_forward_backward(fmm, orc):
    spec = W.WORKLOADS["cube1m_p10"]
    x = W.make("cube1m_p10")
    N = x.shape[0]
    w = W.weights(N, 40)
    T = fmm.Tree(torch.from_numpy(x).cuda(), spec["p"], spec["theta"], spec["ncrit"])
    pot, force = T.evaluate()
    dq, dx = T.backward(torch.from_numpy(w).cuda())
    T.check()
    pg, fg, dqg, dxg = (a.double().cpu().numpy() for a in (pot, force, dq, dx))
    O = orc.OracleTree(x, spec["p"], spec["theta"], spec["ncrit"])
    po, go = O.evaluate()
    assert_match(pg, po, fg, -go, TOL_PHI, TOL_F)
    dqo, dxo = O.backward(w.astype(np.float64))
    assert_match(dqg, dqo, dxg, dxo, TOL_PHI, TOL_F)


def test_cube16m_sampled_parity(fmm, orc):
    spec = W.WORKLOADS["cube16m"]
    x = W.make("cube16m")
    N = x.shape[0]
    assert N == 1 << 24
    idx = W.sample_targets(N, 4096)
    O = orc.OracleTree(x, 8, spec["theta"], spec["ncrit"])
    cases = ((8, False, 4096, 2), (16, False, 1024, 1), (4, True, 4096, 0))
    for p, f64, nt, engine in cases:
        xt = torch.from_numpy(x.astype(np.float64) if f64 else x).cuda()
        T = fmm.Tree(xt, p, spec["theta"], spec["ncrit"])
        assert T.stats()["m2l_engine"] == engine
        pot, force = T.evaluate()
        T.check()
        ii = torch.from_numpy(idx[:nt]).cuda()
        pg = pot[ii].double().cpu().numpy()
        fg = force[ii].double().cpu().numpy()
        T.close()
        del xt, pot, force
        torch.cuda.empty_cache()
        O.set_order(p)
        po, go = O.evaluate(targets=idx[:nt])
        tp, tf = (TOL64_PHI, TOL64_F) if f64 else (TOL_PHI, TOL_F)
        bp, bf = (1e-9, 1e-8) if f64 else (1e-4, 1e-3)
        assert_match(pg, po, fg, -go, tp, tf, bp, bf)


def test_single_tile_fold_accuracy(fmm):
    """At p = 12 (Kp = 144) the M2L runs on the single-tile engine, which adds
    each source entry's TMEM sum into a second accumulator instead of
    accumulating a whole chunk of entries in the tensor core.  The
    single-precision potential then stays within 1.5e-6 (relative L2) of the
    FP64 direct sum on 262,144 cube bodies (6.7e-7 measured; 2.5e-6 with
    16 entries accumulated in TMEM), and the force within 2e-6."""
    from tests.gpu_helpers import rel
    n = 262144
    x = torch.from_numpy(W.cube(n, 2)).cuda()
    idx = torch.from_numpy(W.sample_targets(n, 4096, seed=7).astype(np.int64)).cuda()
    T = fmm.Tree(x, 12, 0.4, 64)
    assert T.stats()["m2l_engine"] == 1
    pot, force = T.evaluate()
    pd, fd = fmm.direct_f64(x, idx)
    torch.cuda.synchronize()
    ii = idx.cpu().numpy()
    pg = pot.cpu().numpy()[ii].astype(np.float64)
    fg = force.cpu().numpy()[ii].astype(np.float64)
    assert rel(pg, pd.cpu().numpy()) < 1.5e-6
    assert rel(fg, fd.cpu().numpy()) < 2e-6
    T.check()
    T.close()
