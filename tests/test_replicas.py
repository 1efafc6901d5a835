"""The multi-GPU path of bench.py, on CPU: two gloo ranks.

The method shards into independent replicas: every rank steps its own particles, with no
collective on the data path. So what N > 1 adds is host logic:
  * the barrier around a timed region;
  * the max of the region's duration over ranks;
  * the whole-job rate, every rank's particle-steps over the slowest rank's time;
  * a distinct seed for each rank's replica;
  * a line printed by rank 0 alone (the reference arm on rank 0 only).
These run here as two processes on the gloo backend, rendezvous on 127.0.0.1.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    ranks = bench.Ranks(backend="gloo", device="cpu")
    try:
        assert (ranks.rank, ranks.world) == (rank, world)
        ranks.barrier()
        # each rank's own "duration"; every rank must see the largest
        got = ranks.max(10.0 + 5.0 * rank)
        ranks.barrier()
        wl = bench.make_workload("weibel128", rank)
        out[rank] = (got, float(wl.x[:16].sum()), wl.n)
    finally:
        ranks.close()


def test_barrier_and_max_over_two_gloo_ranks():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    assert sorted(res) == [0, 1]
    # both ranks hold the max of 10 and 15
    assert res[0][0] == res[1][0] == 15.0
    # replicas: the same size, their own particles
    assert res[0][2] == res[1][2]
    assert res[0][1] != res[1][1]


def test_whole_job_rate_counts_every_rank_over_the_slowest():
    # 2 ranks x 1,048,576 particles x 100 steps in the slowest rank's 9 ms
    v = bench.whole_job_rate(1048576, 2, 100, 9.0)
    assert v == pytest.approx(2 * 1048576 * 100 / 9e-3, rel=1e-15)
    assert bench.whole_job_rate(1048576, 1, 100, 9.0) == pytest.approx(v / 2)


def test_single_rank_needs_no_process_group(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    r = bench.Ranks(backend="gloo", device="cpu")
    assert r.dist is None and (r.rank, r.world) == (0, 1)
    r.barrier()
    assert r.max(3.5) == 3.5
    r.close()


@pytest.mark.slow
def test_reference_arm_prints_on_rank_zero_only():
    # torchrun with two ranks: rank 0 times the oracle and prints the line; rank 1 exits 0
    # without work (a two-step sample keeps this to a few seconds of oracle time)
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--workload", "weibel128", "--steps", "2", "--warmup", "0"]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, env=env, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0
    assert np.isfinite(line["value"])
