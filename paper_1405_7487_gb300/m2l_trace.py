"""Where the tensor-core M2L's time goes: builds the trace variant of the
library (libgbfmm_traced.so, -DGBFMM_M2L_TRACE), runs one evaluation of a
cube workload and prints, per role of the four-tile M2L block, the cycles
spent in each wait and in issuing MMAs, averaged per block.

  python -m paper_1405_7487_gb300.m2l_trace [N] [p]
"""

from __future__ import annotations

import ctypes
import os
import sys

SLOTS = {0: "producers: wait free source stage", 1: "producers: wait free operator stage",
         2: "MMA thread: block start to loop", 3: "MMA thread: loop end to block end",
         5: "MMA: wait operator stage", 6: "MMA: wait source stage", 7: "MMA: issue + commit",
         11: "whole block", 13: "producers: wait last MMA", 14: "epilogue"}


def main(argv):
    n = int(argv[1]) if len(argv) > 1 else 1 << 20
    p = int(argv[2]) if len(argv) > 2 else 10
    os.environ["GBFMM_TRACE"] = "1"
    import numpy as np
    import torch
    from paper_1405_7487_gb300 import build_lib
    build_lib.build(traced=True)
    from paper_1405_7487_gb300 import fmm as F
    from paper_1405_7487_gb300 import workloads as W
    x = torch.from_numpy(W.cube(n, 2)).cuda()
    T = F.Tree(x, p, 0.4, 64, F.FMM_FLAG_TIMING | F.FMM_FLAG_SERIAL_PHASES)
    out = np.zeros(16, np.int64)
    L = F.lib()
    T.evaluate()
    torch.cuda.synchronize()
    L.fmm_debug_m2l_trace(out.ctypes.data_as(ctypes.c_void_p))  # drop the first (cold) pass
    T.evaluate()
    torch.cuda.synchronize()
    if L.fmm_debug_m2l_trace(out.ctypes.data_as(ctypes.c_void_p)) != 1:
        raise SystemExit("not a trace build")
    blocks = max(int(out[12]), 1)
    st = T.stats()
    print(f"N = {n}, p = {p}: M2L {st['ms']['m2l']:.3f} ms (trace build), {blocks} blocks, engine {st['m2l_engine']}")
    for k, name in SLOTS.items():
        print(f"  {name:36s} {out[k] / blocks:12.0f} cycles per block")


if __name__ == "__main__":
    main(sys.argv)
