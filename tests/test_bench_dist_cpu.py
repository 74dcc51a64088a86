"""The N > 1 reporting path of bench.py on the CPU: two gloo ranks, each
timing its own replica; the job's time is the slowest rank's and its rate
counts the cell updates of all ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [10.0 + rank, 2.0 - rank]        # per-rank kernel ms and e2e s
        got = bench._max_over_ranks(dist, mine, "cpu")
        out[rank] = (got, bench._job_rate(1000, 50, world, got[0] * 1e-3))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_report_the_slowest_rank_and_all_work():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, join=True,
                           start_method="spawn")
        res = dict(out)
    for r in (0, 1):
        got, rate = res[r]
        assert got == [11.0, 2.0]
        assert rate == pytest.approx(1000 * 50 * 2 / 11e-3 / 1e6)


def test_single_process_is_the_identity():
    assert bench._max_over_ranks(None, [3.0, 4], "cpu") == [3.0, 4.0]
    assert bench._job_rate(65536, 300, 1, 0.366) == pytest.approx(65536 * 300 / 0.366 / 1e6)


def test_reference_arm_prints_one_json_line_of_the_contract():
    """bench.py --impl reference times the oracle on the host cores and prints
    one JSON line with the arm's metric, unit and configuration, its CPU
    baseline and an end-to-end figure with no device copies."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    for k in ("value", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling", "dtype",
              "data", "config"):
        assert k in line, k
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 3
    assert line["config"]["workload"] == bench.WORKLOAD
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
