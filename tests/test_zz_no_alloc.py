"""The allocation-free entry point fmm_root_keys_noalloc, through the C ABI.

Some callers of this library may not allocate device memory while they call
it: code under a fixed device-memory budget or inside another framework's
allocator, and code that must not risk the device-wide synchronisation a
cudaMalloc/cudaFree can cause.  fmm_root_keys_noalloc serves them: it
computes the root cube and Morton keys of fmm_build's first step with its
scratch in a fixed device array.  This test checks it against the existing
path (fmm_build, then fmm_get_root and fmm_get_keys) bit for bit, on two
calls in a row, checks that repeated calls leave the device's free memory
unchanged, and covers the case where the caller passes no flag word (the
flag then goes to the scratch array).  The file name keeps it last in
collection order.
"""

import ctypes

import numpy as np
import pytest
import torch

from paper_1405_7487_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_1405_7487_gb300 import build_lib
    build_lib.build()
    from paper_1405_7487_gb300 import fmm
    L = fmm.lib()
    L.fmm_root_keys_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]
    L.fmm_root_keys_noalloc.restype = ctypes.c_int
    return fmm


def _call(F, x, root, keys, flag):
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    return F.lib().fmm_root_keys_noalloc(p(x), x.shape[0], p(root), p(keys), p(flag), s)


def test_noalloc_matches_build_twice(F):
    inputs = [W.cube(300000, 91), W.plummer(200000, 92)]
    for x_h in inputs:
        x = torch.from_numpy(x_h).cuda()
        n = x.shape[0]
        T = F.Tree(x, 4, 0.4, 64)
        ref = T.root()
        ks, perm = T.keys()
        ref_keys = np.empty(n, np.uint64)
        ref_keys[perm] = ks
        root = torch.empty(13, dtype=torch.float64, device="cuda")
        keys = torch.empty(n, dtype=torch.int64, device="cuda")
        flag = torch.full((1,), 7, dtype=torch.int32, device="cuda")
        for _ in range(2):  # two calls in a row share the scratch array
            root.fill_(-1.0)
            keys.fill_(-1)
            assert _call(F, x, root, keys, flag) == 0
            torch.cuda.synchronize()
            r = root.cpu().numpy()
            assert np.array_equal(r[0:3], ref["lo"]) and np.array_equal(r[3:6], ref["hi"])
            assert np.array_equal(r[6:9], ref["centre"]) and r[9] == ref["H"]
            assert np.array_equal(r[10:13], ref["corner"])
            assert np.array_equal(keys.cpu().numpy().view(np.uint64), ref_keys)
            assert int(flag.item()) == 0
        T.close()


def test_noalloc_flags_and_limits(F):
    x = torch.from_numpy(W.cube(5000, 93)).cuda()
    x[17, 2] = float("nan")
    root = torch.empty(13, dtype=torch.float64, device="cuda")
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert _call(F, x, root, None, flag) == 0
    torch.cuda.synchronize()
    assert int(flag.item()) == 1
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    big = F.lib().fmm_root_keys_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_int64(1 << 31),
                                        ctypes.c_void_p(root.data_ptr()), None, None, s)
    assert big == -1
    assert b"maximum" in F.lib().fmm_last_error()


def test_noalloc_allocates_nothing(F):
    """After a first call (which looks up the scratch array), further calls
    leave the device's free memory exactly as it was."""
    x = torch.from_numpy(W.cube(400000, 94)).cuda()
    n = x.shape[0]
    root = torch.empty(13, dtype=torch.float64, device="cuda")
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert _call(F, x, root, keys, flag) == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        assert _call(F, x, root, keys, flag) == 0
        assert _call(F, x, root, keys, None) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_keys_without_flag(F):
    """keys requested, no flag word: the keys are still fmm_build's."""
    x_h = W.plummer(150000, 95)
    x = torch.from_numpy(x_h).cuda()
    n = x.shape[0]
    T = F.Tree(x, 4, 0.5, 32)
    ks, perm = T.keys()
    ref_keys = np.empty(n, np.uint64)
    ref_keys[perm] = ks
    ref = T.root()
    root = torch.empty(13, dtype=torch.float64, device="cuda")
    keys = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    for _ in range(2):
        assert _call(F, x, root, keys, None) == 0
        torch.cuda.synchronize()
        assert np.array_equal(keys.cpu().numpy().view(np.uint64), ref_keys)
        r = root.cpu().numpy()
        assert r[9] == ref["H"] and np.array_equal(r[10:13], ref["corner"])
    T.close()
