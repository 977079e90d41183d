"""Host logic of the bench's multi-rank run, on CPU with the gloo backend.

The time step does not shard without a halo exchange, so N GPUs run N
independent replicas: each rank times its own steps, the job's time is the
slowest rank's, and the reported value is the cell-steps of all ranks over that
time. These tests run that reduction in two gloo processes (no GPU), and check
that the reference arm does its work on rank 0 only.
"""
import argparse
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica(rank, world, port, times_ms, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(times_ms[rank], dist, "cpu")
        q.put((rank, ms, bench.job_rate(1000, 10, world, ms / 1000.0)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("times_ms", [(12.5, 17.25), (30.0, 4.0)])
def test_two_replicas_report_the_slowest_rank_and_the_whole_job(times_ms):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_replica, args=(r, 2, port, times_ms, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=120) for _ in range(2))
    finally:
        for p in procs:
            p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0, 0]
    slowest = max(times_ms)
    for rank, (r, ms, v) in enumerate(got):
        assert r == rank
        assert ms == slowest                       # every rank agrees on the job's time
        assert v == pytest.approx(2 * 1000 * 10 / (slowest / 1000.0))   # cells of both replicas


def test_single_rank_reduction_is_the_identity():
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
    assert bench.job_rate(16, 4, 1, 2.0) == 32.0


def test_reference_arm_runs_on_rank_zero_only(capsys):
    args = argparse.Namespace(gpus=2, steps=1, warmup=0, workload="tgv256", precision=None)
    assert bench.run_reference(args, rank=1, world=2) == 0
    assert capsys.readouterr().out == ""


def test_gpus_must_match_the_process_count():
    # --gpus N is N processes under torchrun; one process asked for two GPUs
    # refuses (exit 2) before it touches a GPU or the oracle
    import subprocess
    import sys
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--gpus", "2", "--impl", "reference"], cwd=root, env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 2 and "WORLD_SIZE" in r.stderr, (r.returncode, r.stderr[-300:])


def test_reference_arm_prints_one_contract_line():
    # the oracle arm on the host cores prints one JSON line with the keys the
    # bench contract asks for, on the default workload's bounded sample
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["dtype"] == "f64" and d["config"]["workload"].startswith("msphere3d 512x256x256")
    # value is the sample's cell-steps over the timed seconds
    assert d["value"] * d["ms_per_step"] / 1000.0 == pytest.approx(128 * 64 * 64, rel=1e-9)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and "128x64x64" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
