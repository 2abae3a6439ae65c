"""Host-side checks of the C ABI library (no GPU needed, no compute calls)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbfmm.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fmm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1405_7487_gb300 import build_lib
    return build_lib.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("fmm_build", "fmm_evaluate", "fmm_backward", "fmm_destroy", "fmm_get_stats", "fmm_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    for n in declared_functions():
        assert hasattr(L, n), n


def test_strerror_without_gpu(libpath):
    L = ctypes.CDLL(libpath)
    L.fmm_strerror.restype = ctypes.c_char_p
    assert L.fmm_strerror(0) == b"ok"
    assert b"argument" in L.fmm_strerror(-1)


def test_null_arguments_rejected_before_any_gpu_work(libpath):
    L = ctypes.CDLL(libpath)
    h = ctypes.c_void_p()
    assert L.fmm_build(None, ctypes.c_int64(10), 4, ctypes.c_double(0.4), 8, 0, None, None, ctypes.byref(h)) == -1
    assert L.fmm_destroy(None) == 0


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1405_7487_gb300 import fmm
    monkeypatch.setattr(fmm, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(fmm, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        fmm.lib()


def test_product_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1405_7487_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "fmm_oracle" not in txt, f


def test_build_arguments_checked_before_any_gpu_work(libpath):
    # every rejected argument returns FMM_ERR_ARG (-1) before a CUDA call, so
    # this runs without a GPU; the position pointer is never dereferenced
    L = ctypes.CDLL(libpath)
    dummy = ctypes.c_void_p(16)
    h = ctypes.c_void_p(1)
    ok = dict(n=1000, p=4, theta=0.4, ncrit=8, flags=0)
    bad = [dict(n=0), dict(n=1 << 31), dict(p=0), dict(p=17), dict(theta=0.0), dict(theta=1.0),
           dict(theta=float("nan")), dict(theta=-0.5), dict(ncrit=0), dict(flags=1 << 8),
           dict(flags=1 << 31)]
    for b in bad:
        a = dict(ok, **b)
        for build in (L.fmm_build, L.fmm_build_f64):
            h.value = 1
            rc = build(dummy, ctypes.c_int64(a["n"]), a["p"], ctypes.c_double(a["theta"]), a["ncrit"],
                       ctypes.c_uint32(a["flags"]), None, None, ctypes.byref(h))
            assert rc == -1, b
            assert not h.value  # the handle is cleared on failure

    class Alloc(ctypes.Structure):
        _fields_ = [("alloc", ctypes.c_void_p), ("free", ctypes.c_void_p), ("ctx", ctypes.c_void_p)]

    half = Alloc(ctypes.c_void_p(16), None, None)  # an allocator without a free function
    assert L.fmm_build(dummy, ctypes.c_int64(1000), 4, ctypes.c_double(0.4), 8, ctypes.c_uint32(0),
                       ctypes.byref(half), None, ctypes.byref(h)) == -1
    # null handles and outputs
    assert L.fmm_evaluate(None, None, dummy, None, None) == -1
    assert L.fmm_backward(None, dummy, dummy, dummy, None) == -1
    assert L.fmm_solve_host(None, None, ctypes.c_int64(10), 4, ctypes.c_double(0.4), 8, ctypes.c_uint32(0),
                            dummy, None, None, None, None) == -1


def test_binding_rejects_bad_shapes_before_the_library(libpath):
    # checked in Python before any library call, so no GPU is needed
    import numpy as np
    import torch

    from paper_1405_7487_gb300 import fmm
    with pytest.raises(ValueError):
        fmm.Tree(torch.zeros(10, 4), 4, 0.4, 8)  # a host tensor
    with pytest.raises(ValueError):
        fmm.solve_host(np.zeros((10, 3), np.float32), None, 4, 0.4, 8)
    with pytest.raises(ValueError):
        fmm.solve_host(np.zeros((0, 4), np.float32), None, 4, 0.4, 8)
    with pytest.raises(ValueError):
        fmm.solve_host(np.zeros((10, 4), np.float32), np.zeros(9, np.float32), 4, 0.4, 8)
    with pytest.raises(TypeError):
        fmm.direct_f64(torch.zeros(10, 4), torch.zeros(3, dtype=torch.int64))


C_CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "gbfmm.h"

int main(void) {
  fmm_tree* t = (fmm_tree*)1;
  int rc = fmm_build(NULL, 10, 4, 0.4, 8, 0u, NULL, NULL, &t);
  if (rc != FMM_ERR_ARG || t != NULL) return 1;
  if (strcmp(fmm_strerror(FMM_ERR_ARG), fmm_strerror(FMM_OK)) == 0) return 2;
  if (fmm_destroy(NULL) != FMM_OK) return 3;
  if (fmm_launch_count() != 0) return 4;
  printf("%s\n", fmm_strerror(rc));
  return 0;
}
"""


def test_plain_c_client_compiles_links_and_runs(libpath, tmp_path):
    # the boundary is a C ABI: a C99 program includes the header, links the
    # library and calls it (argument checks only, so no GPU is needed)
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    libdir = os.path.dirname(libpath)
    name = os.path.basename(libpath)
    assert name.startswith("lib") and name.endswith(".so")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe), "-L", libdir, "-l" + name[3:-3], "-Wl,-rpath," + libdir],
                   check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.strip() == "invalid argument"


def test_stats_struct_layout_matches_header(tmp_path):
    """The binding's fmm_stats mirror has the header's size and field offsets
    (a C program prints them)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    from paper_1405_7487_gb300 import fmm
    names = [n for n, _ in fmm.Stats._fields_]
    prog = "#include <stdio.h>\n#include <stddef.h>\n#include \"gbfmm.h\"\nint main(void) {\n"
    prog += '  printf("%zu\\n", sizeof(fmm_stats));\n'
    for n in names:
        prog += '  printf("%zu\\n", offsetof(fmm_stats, ' + n + '));\n'
    prog += "  return 0;\n}\n"
    src = tmp_path / "layout.c"
    src.write_text(prog)
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    out = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert out[0] == ctypes.sizeof(fmm.Stats)
    assert out[1:] == [getattr(fmm.Stats, n).offset for n in names]
