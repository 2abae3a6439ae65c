"""Host logic of bench.py's multi-rank mode (replicas only), on CPU with gloo.

Every rank runs an independent replica, and the only cross-rank steps are a
barrier and the max-reduction of the timed seconds.  These tests run two
gloo ranks on the host and check that reduction and the whole-job
throughput formula.
"""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r "took" 1 + r seconds: the job time is the slowest rank's
        mx = bench.reduce_max(1.0 + rank, "cpu")
        v = bench.aggregate(1000, 5, world, mx)
        dist.barrier()
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{mx} {v}\n")
    finally:
        dist.destroy_process_group()


def test_reduce_max_and_aggregate_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        mx, v = map(float, (tmp_path / f"r{r}.txt").read_text().split())
        assert mx == 2.0  # every rank sees the maximum
        assert v == pytest.approx(1000 * 5 * world / 2.0)


def test_single_process_reduce_is_identity():
    assert bench.reduce_max(3.25, "cpu") == 3.25
    assert bench.aggregate(10, 2, 1, 4.0) == 5.0


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    # ranks other than 0 print nothing and touch neither the oracle nor a GPU
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        workload, steps, warmup = "cube4k_p4", 1, 0

    bench.run_reference(A())
    assert capsys.readouterr().out == ""


@pytest.mark.parametrize("mac", ["half", "tight"])
def test_reference_arm_line_on_rank0(monkeypatch, capsys, mac):
    # rank 0 times the oracle on the host and prints one JSON line of the
    # benchmark's schema, with the e2e block of a host-only program
    import json
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")

    class A:
        workload, steps, warmup = "cube4k_p4", 2, 1

    A.mac = mac
    bench.run_reference(A())
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1
    assert d["config"]["workload"] == "cube4k_p4" and d["config"]["N"] == 4096
    assert d["config"].get("mac", "half") == mac
    assert d["ms_per_step"] == pytest.approx(4096 / d["value"] * 1e3)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
