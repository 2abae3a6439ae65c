"""The C ABI's failure and memory paths, and the double-precision direct sum
the accuracy figures come from (all through the library, on the GPU).

* fmm_direct_f64 against the oracle's direct sum (the O(N^2) definition the
  FMM approximates), with coincident bodies and edge indices.
* A caller-supplied stream-ordered allocator: every byte of workspace goes
  through it, the outputs are bit-identical to the library pool's, and the
  allocations are balanced by frees when the tree is destroyed.
* An allocator that fails at its k-th call, for every k a build makes: each
  build returns FMM_ERR_OOM, gives back every byte it took, and the next
  build succeeds.
* A device scan that waits past its limit (the test switch makes the first
  tile publish late): fmm_build returns FMM_ERR_TIMEOUT, gives back its
  memory, and the next build succeeds with the same results as before.
"""

import ctypes

import numpy as np
import pytest
import torch

from paper_1405_7487_gb300 import workloads as W
from tests.gpu_helpers import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fmm():
    from paper_1405_7487_gb300 import build_lib
    build_lib.build()
    from paper_1405_7487_gb300 import fmm as F
    assert torch.cuda.is_available()
    return F


# ------------------------------------------------------------ direct sum

@pytest.mark.parametrize("dist", ["cube", "plummer"])
def test_direct_f64_matches_oracle(fmm, orc, dist):
    """fmm_direct_f64 equals the oracle's double direct sum to 1e-12 (both
    sum the same float32 inputs in double; only the order of the additions
    differs), with coincident bodies (they contribute nothing to each other)
    and the first and last indices among the targets."""
    n = 20000
    x = W.cube(n, 51) if dist == "cube" else W.plummer(n, 52)
    x[1000:1010, :3] = x[7, :3]  # eleven bodies at one point
    idx = np.concatenate([[0, n - 1, 7, 1005], W.sample_targets(n, 1000, seed=53)]).astype(np.int64)
    xt = torch.from_numpy(x).cuda()
    pg, fg = fmm.direct_f64(xt, torch.from_numpy(idx).cuda())
    torch.cuda.synchronize()
    po, go = orc.direct(x, targets=idx)
    pg, fg = pg.cpu().numpy(), fg.cpu().numpy()
    assert rel(pg, po) < 1e-12
    assert rel(fg, -go) < 1e-12
    assert np.max(np.abs(pg - po) / np.maximum(np.abs(po), 1e-300)) < 1e-10
    # a target index outside [0, n) is not a body: NaN, and the others stay put
    bad = torch.tensor([3, -1, n, 5], dtype=torch.int32, device="cuda")
    pb, fb = fmm.direct_f64(xt, bad)
    pb, fb = pb.cpu().numpy(), fb.cpu().numpy()
    assert np.isnan(pb[1]) and np.isnan(pb[2]) and np.all(np.isnan(fb[1:3]))
    po2, _ = orc.direct(x, targets=np.array([3, 5]))
    assert rel(pb[[0, 3]], po2) < 1e-12


# ------------------------------------------------------------- allocator

class Counting:
    """A stream-ordered allocator over torch's caching allocator that counts
    calls and bytes, and can fail (return NULL) at its k-th call."""

    def __init__(self, fail_at: int = 0):
        self.fail_at = fail_at
        self.calls = 0
        self.bytes = 0
        self.live = {}
        self.frees = 0
        self.alloc_fn = fmm_mod().ALLOC_FN(self._alloc)
        self.free_fn = fmm_mod().FREE_FN(self._free)
        self.struct = fmm_mod().Allocator(self.alloc_fn, self.free_fn, None)

    def _alloc(self, size, stream, ctx):
        self.calls += 1
        if self.fail_at and self.calls == self.fail_at:
            return None
        ptr = torch.cuda.caching_allocator_alloc(max(int(size), 1), stream=int(stream or 0))
        self.live[ptr] = int(size)
        self.bytes += int(size)
        return ptr

    def _free(self, ptr, stream, ctx):
        self.frees += 1
        assert ptr in self.live, "free of a pointer this allocator did not hand out"
        del self.live[ptr]
        torch.cuda.caching_allocator_delete(ptr)


def fmm_mod():
    from paper_1405_7487_gb300 import fmm as F
    return F


def outputs(T, w):
    pot, force = T.evaluate()
    dq, dx = T.backward(w)
    torch.cuda.synchronize()
    return [a.cpu().numpy() for a in (pot, force, dq, dx)]


def test_caller_allocator_takes_all_workspace(fmm):
    x = torch.from_numpy(W.plummer(60000, 54)).cuda()
    w = torch.from_numpy(W.weights(60000, 55)).cuda()
    ref = outputs(fmm.Tree(x, 8, 0.5, 32), w)
    A = Counting()
    T = fmm.Tree(x, 8, 0.5, 32, allocator=A.struct)
    got = outputs(T, w)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
    # every byte the tree accounts for came from the caller's allocator
    assert A.bytes == T.stats()["workspace_bytes"] and A.calls > 0
    T.lists()  # the inspection call's workspace goes through it too
    T.close()
    torch.cuda.synchronize()
    assert not A.live and A.frees == A.calls


def test_allocator_failure_at_every_call(fmm):
    """An allocator that returns NULL at call k, for every k up to the number
    of calls one build makes: FMM_ERR_OOM, every byte given back, and a clean
    build afterwards."""
    x = torch.from_numpy(W.cube(20000, 56)).cuda()
    probe = Counting()
    T = fmm.Tree(x, 6, 0.4, 64, allocator=probe.struct)
    ref = outputs(T, torch.ones(20000, device="cuda"))
    T.close()
    n_calls = probe.calls
    assert n_calls > 10
    for k in range(1, n_calls + 1):
        A = Counting(fail_at=k)
        with pytest.raises(fmm.FMMError) as e:
            fmm.Tree(x, 6, 0.4, 64, allocator=A.struct)
        assert e.value.name == "FMM_ERR_OOM", (k, e.value)
        torch.cuda.synchronize()
        assert not A.live, (k, len(A.live))
        assert A.frees == A.calls - 1
    T = fmm.Tree(x, 6, 0.4, 64, allocator=Counting().struct)
    for a, b in zip(outputs(T, torch.ones(20000, device="cuda")), ref):
        assert np.array_equal(a, b)


# ------------------------------------------------------- bounded waits

def test_scan_wait_past_limit_is_timeout(fmm):
    """With the test switch on, the first tile of every multi-tile device
    scan publishes 10 ms late and the look-back's limit is 1 ms: the build
    returns FMM_ERR_TIMEOUT and gives back all its memory.  With the switch
    off again the next build succeeds, with the same results as before."""
    L = fmm.lib()
    n = 300000
    x = torch.from_numpy(W.cube(n, 57)).cuda()
    w = torch.from_numpy(W.weights(n, 58)).cuda()
    ref = outputs(fmm.Tree(x, 6, 0.4, 64), w)
    A = Counting()
    prev = L.fmm_debug_scan_fault(1)
    try:
        with pytest.raises(fmm.FMMError) as e:
            fmm.Tree(x, 6, 0.4, 64, allocator=A.struct)
    finally:
        L.fmm_debug_scan_fault(prev)
    assert e.value.name == "FMM_ERR_TIMEOUT"
    assert b"look-back" in L.fmm_last_error()
    torch.cuda.synchronize()
    assert not A.live and A.calls > 0
    T = fmm.Tree(x, 6, 0.4, 64)
    got = outputs(T, w)
    T.check()
    assert T.stats()["device_errors"] == 0
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


def test_check_after_clean_passes(fmm):
    x = torch.from_numpy(W.cube(5000, 59)).cuda()
    T = fmm.Tree(x, 4, 0.4, 64)
    T.evaluate()
    T.check()
    assert fmm.lib().fmm_check(None) == -1
