"""Benchmark of the GB300 FMM hot path: one JSON line on stdout.

A step is one whole pass of the hot path on one batch of synthetic bodies:
fmm_build (bounding cube, keys, sort, octree, dual traversal, lists,
operators), fmm_evaluate (P2M, M2M, M2L, L2L, P2P, L2P: potential + force)
and fmm_backward (adjoint of sum w_i phi_i), with the inputs resident in HBM.
`value` is particles per second over the whole job (all ranks); `e2e` is
the same through fmm_solve_host with pinned host buffers (copies included).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the double-precision CPU oracle

With N > 1 (torchrun) every rank runs an independent replica (the method is
not sharded across GPUs); the time is the maximum over ranks.

The timed steps run as a user runs them: the near field (P2P) on a second,
lower-priority stream concurrently with the far field, with per-phase CUDA
events on the stream each phase runs on (the roofline's kernel time is the
M2L span measured that way).  Five further steps run the phases one at a
time ("isolated"), each after an L2 flush: per-kernel times without sharing
the GPU, averaged over the five, from which the P2P fraction of the FP32
peak is reported.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "FMM particles/sec (pot+force) at N=1M, rel-L2 err vs FP64 direct; P2P % FP32 peak"
UNIT = "particles/s"
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2
# DRAM bytes (read + write) per launch of the dominant kernel from one ncu
# capture (profiles/k_m2l_tc4_cube1m_p10_dram.md): workload, N, kernel.
# Entries are dropped when the kernel changes.
DRAM_TRAFFIC = {("cube1m_p10", 1048576, "k_m2l_tc4"): 401_603_584 + 601_194_752}
CPU_SAMPLE_N = 65536
ISO_STEPS = 5  # serial-phase steps behind the per-kernel ("isolated") figures


# ------------------------------------------------------------------ helpers

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def reduce_max(x: float, device) -> float:
    """Maximum of a host float over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(n_per_rank: int, steps: int, world: int, max_seconds: float) -> float:
    """Whole-job throughput: all ranks' particles over the slowest rank's time."""
    return n_per_rank * steps * world / max_seconds


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()
        # nvidia-smi takes a while to start: let its first sample arrive, so
        # that the samples cover the timed region that follows
        t_end = time.time() + 3.0
        while not self.lines and time.time() < t_end and self.proc.poll() is None:
            time.sleep(0.01)
        self.lines.clear()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except (OSError, ValueError):
        return {}


# --------------------------------------------------------------- GPU arm

def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    from paper_1405_7487_gb300 import build_lib
    if rank == 0:
        build_lib.build()
    if world > 1:
        dist.barrier()
    from paper_1405_7487_gb300 import fmm as F
    from paper_1405_7487_gb300 import workloads as W

    spec = W.WORKLOADS[args.workload]
    p, theta, ncrit = spec["p"], spec["theta"], spec["ncrit"]
    x_h = W.make(args.workload, n=args.n)
    N = x_h.shape[0]
    w_h = W.weights(N, spec.get("wseed", 40))
    x = torch.from_numpy(x_h).to(dev)
    w = torch.from_numpy(w_h).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    extra = F.FMM_FLAG_MUTUAL_P2P if args.p2p == "mutual" else 0
    extra |= {"half": 0, "circ": F.FMM_FLAG_CIRCUMSCRIBED, "tight": F.FMM_FLAG_TIGHT_MAC,
              "fitted": F.FMM_FLAG_FITTED_CENTRES}[args.mac]

    def step(flags=F.FMM_FLAG_TIMING):
        T = F.Tree(x, p, theta, ncrit, flags | extra)
        pot, force = T.evaluate()
        dq, dx = T.backward(w)
        st = T.stats()
        T.close()
        return st, pot, force

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    step_ms, m2l_ms, p2p_ms, stats = [], [], [], None
    launches0 = F.launch_count()
    for _ in range(args.steps):
        flush.zero_()  # L2 flush between timed steps (not timed)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats, pot, force = step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        m2l_ms.append(stats["ms"]["m2l"])
        p2p_ms.append(stats["ms"]["p2p"])
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    launches = F.launch_count() - launches0
    clk = clocks.stop()
    total_s = sum(step_ms) / 1e3
    max_s = reduce_max(total_s, dev)
    value = aggregate(N, args.steps, world, max_s)

    # the same step with the phases run one at a time (ISO_STEPS steps, after
    # the timed region, each after an L2 flush): per-kernel times without the
    # near field sharing the GPU, averaged over the steps
    iso_ms = []
    for _ in range(ISO_STEPS):
        flush.zero_()
        st_iso, _, _ = step(F.FMM_FLAG_TIMING | F.FMM_FLAG_SERIAL_PHASES)
        iso_ms.append(st_iso["ms"])
    iso = {"ms": {k: statistics.mean(m[k] for m in iso_ms) for k in iso_ms[0]}}

    # accuracy against the double direct sum on 4096 sampled targets
    idx = torch.from_numpy(W.sample_targets(N, 4096)).to(dev)
    pd, fd = F.direct_f64(x, idx)
    ii = idx.long()
    err_pot = float(torch.linalg.norm(pot[ii].double() - pd) / torch.linalg.norm(pd))
    err_force = float(torch.linalg.norm(force[ii].double() - fd) / torch.linalg.norm(fd))

    # end to end through host buffers (pinned), copies inside the timed region
    xh = torch.from_numpy(x_h).pin_memory().numpy()
    wh = torch.from_numpy(w_h).pin_memory().numpy()
    F.solve_host(xh, wh, p, theta, ncrit, flags=extra)
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        F.solve_host(xh, wh, p, theta, ncrit, flags=extra)
    e2e_s = reduce_max(time.perf_counter() - t0, dev)
    e2e = {"value": aggregate(N, args.steps, world, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": int(x_h.nbytes + w_h.nbytes),
           "d2h_bytes_per_step": int(N * 4 + N * 12 + N * 4 + N * 12)}

    # roofline of the dominant kernel (both are FP32 ALU bound)
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = clk["sm_mhz"] or measured_peaks().get("sm_max_mhz", 2070.0)
    fp32_peak_tflops = props.multi_processor_count * 128 * 2 * sm_mhz * 1e6 / 1e12
    m2l_avg = statistics.mean(m2l_ms)
    p2p_avg = statistics.mean(p2p_ms)
    K = stats["K"]
    p2p_flops = 20.0 * stats["n_p2p_body_pairs"]
    m2l_flops = 2.0 * K * K * stats["n_m2l"]
    p2p_tf = p2p_flops / (p2p_avg * 1e-3) / 1e12
    m2l_tf = m2l_flops / (m2l_avg * 1e-3) / 1e12
    p2p_tf_iso = p2p_flops / (iso["ms"]["p2p"] * 1e-3) / 1e12
    m2l_tf_iso = m2l_flops / (iso["ms"]["m2l"] * 1e-3) / 1e12
    # TF32 dense tensor peak: the measured bf16 burst x the nominal tf32/bf16
    # ratio (1.1 / 2.25 PFLOP/s)
    mp = measured_peaks()
    tf32_peak_tflops = mp.get("bf16_tflops", 1900.0) * (1.1 / 2.25)
    # the dominant kernel by its time alone (in the timed steps P2P's span
    # stretches under M2L, which it runs beside)
    if iso["ms"]["m2l"] >= iso["ms"]["p2p"]:
        if stats["m2l_engine"] in (1, 2):
            kname = "k_m2l_tc4" if stats["m2l_engine"] == 2 else "k_m2l_tc"
            dom = {"kernel": f"{kname} (+k_split_tf32, reduce)", "bound": "tensor", "achieved": m2l_tf,
                   "ms": m2l_avg, "traffic": DRAM_TRAFFIC.get((args.workload, N, kname)),
                   "peak": tf32_peak_tflops,
                   "peak_source": "measured bf16 dense burst (MEASURED_PEAKS.json) x 1.1/2.25 (nominal tf32/bf16)"}
        else:
            dom = {"kernel": "k_m2l_cc", "bound": "alu", "achieved": m2l_tf, "ms": m2l_avg,
                   "peak": fp32_peak_tflops,
                   "peak_source": "FP32 spec formula SMs x 128 lanes x 2 x median SM clock under load"}
    else:
        dom = {"kernel": "k_p2p", "bound": "alu", "achieved": p2p_tf, "ms": p2p_avg, "peak": fp32_peak_tflops,
               "peak_source": "FP32 spec formula SMs x 128 lanes x 2 x median SM clock under load"}
    roofline = {"bound": dom["bound"], "kernel": dom["kernel"], "achieved": round(dom["achieved"], 3),
                "peak": round(dom["peak"], 3), "unit": "TFLOP/s",
                "frac": round(dom["achieved"] / dom["peak"], 4), "traffic": dom.get("traffic"),
                "peak_source": dom["peak_source"], "avg_launch_ms": round(dom["ms"], 4),
                "work": "algorithmic: 2 K^2 flops per M2L pair (K = p^2), 20 flops per P2P body pair"}
    slots = stats["n_m2l_slots"]
    Kp = (K + 15) // 16 * 16
    m2l_exec_flops = 3 * 2.0 * slots * Kp * Kp if stats["m2l_engine"] in (1, 2) else 2.0 * slots * Kp * Kp

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_s * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "distribution": spec["dist"], "N": N, "p": p, "theta": theta,
                   "ncrit": ncrit, "step": "fmm_build + fmm_evaluate (pot, force) + fmm_backward",
                   "l2": "flushed between timed steps (512 MiB write)", "parallelism": f"replicas x{world}",
                   **({"p2p": "mutual"} if args.p2p == "mutual" else {}),
                   **({"mac": args.mac} if args.mac != "half" else {})},
        "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline,
        "p2p_frac_fp32_peak": round(p2p_tf_iso / fp32_peak_tflops, 4),
        # P2P span in the timed steps, where it shares the GPU with M2L
        "p2p_frac_fp32_peak_in_step": round(p2p_tf / fp32_peak_tflops, 4),
        "m2l_tflops": round(m2l_tf, 3), "p2p_tflops": round(p2p_tf, 3),
        "isolated": {"steps": ISO_STEPS, "m2l_tflops": round(m2l_tf_iso, 3), "p2p_tflops": round(p2p_tf_iso, 3),
                     "m2l_frac": round(m2l_tf_iso / dom["peak"], 4) if dom["bound"] == "tensor" else None,
                     "phase_ms": {k: round(v, 4) for k, v in iso["ms"].items()}},
        "m2l_issued_tflops": round(m2l_exec_flops / (m2l_avg * 1e-3) / 1e12, 3),
        "eval_only_particles_per_s": N / (stats["ms"]["eval_total"] * 1e-3),
        "err_vs_direct": {"pot": err_pot, "force": err_force, "targets": 4096},
        "phase_ms": {k: round(v, 4) for k, v in stats["ms"].items()},
        "tree": {k: stats[k] for k in ("n_cells", "n_leaves", "n_levels", "n_m2l", "n_p2p_body_pairs",
                                       "n_m2l_classes", "n_m2l_tiles", "n_m2l_slots", "m2l_engine",
                                       "workspace_bytes", "device_errors")},
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload, steps=1, mac=args.mac)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------- oracle (CPU)

def cpu_baseline(workload: str, steps: int, mac: str = "half") -> dict:
    """The double-precision oracle, as it stands, on the host cores: a bounded
    sample (the first CPU_SAMPLE_N bodies of the same workload, same p, theta,
    ncrit and MAC radius); each step = oracle build + forward + backward."""
    import numpy as np

    import oracle
    from paper_1405_7487_gb300 import workloads as W
    spec = W.WORKLOADS[workload]
    oracle.build()
    cores = oracle.set_threads(0)
    x = W.make(workload)[:CPU_SAMPLE_N]
    w = W.weights(x.shape[0], spec.get("wseed", 40)).astype(np.float64)
    t0 = time.perf_counter()
    for _ in range(steps):
        T = oracle.OracleTree(x, spec["p"], spec["theta"], spec["ncrit"], circumscribed=mac == "circ",
                              tight=mac == "tight", fitted=mac == "fitted")
        T.backward(w)  # evaluates with q (forward) and with w (adjoint)
        del T
    dt = time.perf_counter() - t0
    return {"value": x.shape[0] * steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "bodies": int(x.shape[0]),
            "sample": f"first {x.shape[0]} bodies of {workload}, same p/theta/ncrit"
                      f"{'' if mac == 'half' else ', ' + mac + ' MAC radius'}; "
                      f"build + forward + backward, {steps} step(s), {dt:.2f} s"}


# ------------------------------------------------- precision / scale sweep

def run_sweep(args):
    """The precision and scale sweep: N bodies of the cube16m workload
    (16,777,216 by default), p in {4, 8, 12, 16}.  The single-precision path
    (FP32 P2P with compensation, 3xTF32 M2L) and the all-double path each run
    build + forward + backward, timed with CUDA events after one warm-up step,
    and their errors against the double direct sum on 4,096 sampled targets
    are measured.  One JSON line per (p, path), then one line comparing the
    paths at matched error: for each error level both paths reach, the time
    of each, interpolated log-linearly between neighbouring p."""
    import math

    import numpy as np
    import torch
    from paper_1405_7487_gb300 import build_lib
    build_lib.build()
    from paper_1405_7487_gb300 import fmm as F
    from paper_1405_7487_gb300 import workloads as W

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    spec = W.WORKLOADS["cube16m"]
    x_h = W.make("cube16m", n=args.n)
    N = x_h.shape[0]
    w_h = W.weights(N, 41)
    x32 = torch.from_numpy(x_h).to(dev)
    idx = torch.from_numpy(W.sample_targets(N, 4096)).to(dev)
    pd, fd = F.direct_f64(x32, idx)
    ii = idx.long()
    stream = torch.cuda.current_stream(dev)
    rows = []
    for p in spec["p"]:
        for prec in ("f32", "f64"):
            if prec == "f64" and p > args.sweep_max_p_f64:
                continue
            dt = torch.float32 if prec == "f32" else torch.float64
            x = x32.to(dt)
            w = torch.from_numpy(w_h).to(dev, dt)

            def step():
                T = F.Tree(x, p, spec["theta"], spec["ncrit"], F.FMM_FLAG_TIMING)
                pot, force = T.evaluate()
                T.backward(w)
                st = T.stats()
                T.close()
                return pot, force, st

            step()
            torch.cuda.synchronize(dev)
            times = []
            for _ in range(args.steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pot, force, st = step()
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
            err_p = float(torch.linalg.norm(pot[ii].double() - pd) / torch.linalg.norm(pd))
            err_f = float(torch.linalg.norm(force[ii].double() - fd) / torch.linalg.norm(fd))
            row = {"sweep": "precision", "N": N, "p": p, "path": prec, "ms_per_step": statistics.mean(times),
                   "step": "fmm_build + fmm_evaluate + fmm_backward", "err_vs_direct": {"pot": err_p, "force": err_f},
                   "phase_ms": {k: round(v, 3) for k, v in st["ms"].items()}, "m2l_engine": st["m2l_engine"],
                   "n_m2l": st["n_m2l"], "n_p2p_body_pairs": st["n_p2p_body_pairs"]}
            rows.append(row)
            print(json.dumps(row), flush=True)
            del pot, force
            torch.cuda.empty_cache()

    def at_error(path, e):
        pts = sorted((r["p"], r["err_vs_direct"]["pot"], r["ms_per_step"]) for r in rows if r["path"] == path)
        for (p0, e0, t0), (p1, e1, t1) in zip(pts, pts[1:]):
            if (e0 - e) * (e1 - e) <= 0 and e0 != e1:
                u = (math.log(e) - math.log(e0)) / (math.log(e1) - math.log(e0))
                return math.exp(math.log(t0) + u * (math.log(t1) - math.log(t0)))
        for pp, ee, tt in pts:  # exactly reached at a measured p
            if ee == e:
                return tt
        return None

    cmp = {}
    for e in (1e-2, 1e-3, 1e-4, 1e-5, 1e-6):
        a, b = at_error("f32", e), at_error("f64", e)
        if a is not None and b is not None:
            cmp[f"{e:.0e}"] = {"f32_ms": round(a, 2), "f64_ms": round(b, 2), "f64_over_f32": round(b / a, 2)}
    print(json.dumps({"sweep": "precision", "N": N, "matched_error": cmp}), flush=True)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_1405_7487_gb300 import workloads as W
    spec = W.WORKLOADS[args.workload]
    for _ in range(args.warmup):
        cpu_baseline(args.workload, 1, args.mac)
    cb = cpu_baseline(args.workload, args.steps, args.mac)
    out = {"metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": cb["bodies"] / cb["value"] * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": args.workload, "distribution": spec["dist"], "N": cb["bodies"],
                      "p": spec["p"], "theta": spec["theta"], "ncrit": spec["ncrit"],
                      "step": "oracle build + forward + backward"},
           "cpu_baseline": cb,
           "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if args.mac != "half":
        out["config"]["mac"] = args.mac
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbfmm", choices=["gbfmm", "reference"])
    ap.add_argument("--workload", default="cube1m_p10")
    ap.add_argument("--n", type=int, default=None, help="bodies (default: the workload's size)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep", default=None, choices=["precision"],
                    help="precision/scale sweep (cube16m: FP32 vs all-FP64 at p = 4..16), JSON lines")
    ap.add_argument("--sweep-max-p-f64", type=int, default=16, help="largest p of the double path in the sweep")
    ap.add_argument("--mac", default="half", choices=["half", "circ", "tight", "fitted"],
                    help="MAC radius: half side of the cube (default), half diagonal, particle-fitted; "
                         "fitted: expansion centres and radii fitted to the bodies")
    ap.add_argument("--p2p", default="one-sided", choices=["one-sided", "mutual"],
                    help="near field: one block per target leaf, or mutual interaction")
    args = ap.parse_args()
    if args.sweep == "precision":
        run_sweep(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
