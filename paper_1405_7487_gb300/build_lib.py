"""Compile the CUDA library ``libgbfmm.so`` in-tree for sm_103a.

Each ``csrc/*.cu`` is compiled to an object in parallel with ``nvcc`` and the
objects are linked into a shared library next to this file.  Objects go to
``_build/`` under the package (git-ignored).  Nothing is downloaded and no
build system beyond nvcc is needed.
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(PKG, "libgbfmm.so")
BUILD = os.path.join(PKG, "_build")
CHECKED_OUT = os.path.join(PKG, "libgbfmm_checked.so")
TRACED_OUT = os.path.join(PKG, "libgbfmm_traced.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgbfmm.so")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps_mtime() -> float:
    files = sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    files.append(os.path.join(INCLUDE, "gbfmm.h"))
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, extra=(), checked: bool = False,
          traced: bool = False) -> str:
    """Build (if stale) and return the path of libgbfmm.so.

    checked=True builds libgbfmm_checked.so instead: the evaluation kernels
    bounds-check their data-dependent accesses (see fmm_debug_checks).
    traced=True builds libgbfmm_traced.so: the tensor-core M2L counts the
    cycles of each role's waits and work (see fmm_debug_m2l_trace)."""
    out_path = CHECKED_OUT if checked else (TRACED_OUT if traced else OUT)
    if checked:
        extra = tuple(extra) + ("-DGBFMM_CHECKED",)
    if traced:
        extra = tuple(extra) + ("-DGBFMM_M2L_TRACE",)
    if not force and os.path.exists(out_path) and os.path.getmtime(out_path) >= _deps_mtime():
        return out_path
    bdir = BUILD + ("_checked" if checked else ("_traced" if traced else ""))
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = out_path + f".{os.getpid()}.tmp"
    cmd = [cc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out_path)
    return out_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv,
                traced="--traced" in sys.argv))
