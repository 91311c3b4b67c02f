"""The multi-process (replica) path of bench.py, run on the CPU with the gloo backend.

The solver has no exchange step: with N GPUs each rank solves its own seeded replica of the
workload, the step time is the slowest rank's (max over ranks), and the job's rate is N replicas'
nodes over that time.  These tests run that host logic in two gloo processes, and the reference arm
under torchrun, where rank 0 alone times the oracle and prints the line.
"""
import importlib.util
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        w, r, _ = b.dist_env()
        ms = b.max_over_ranks(100.0 * (rank + 1), "cpu")  # rank 1 is the slow one
        out[rank] = (w, r, ms, b.whole_job_rate(w, 1000, ms), b.replica_seed(r))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_with_gloo():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank, (w, r, ms, rate, seed) in res.items():
        assert (w, r) == (2, rank)
        assert ms == 200.0                       # the slowest rank's time on every rank
        assert rate == pytest.approx(2 * 1000 / 0.2)
    assert res[0][4] != res[1][4]                # distinct replicas


def test_single_process_needs_no_group():
    b = _bench()
    assert b.max_over_ranks(3.5, "cpu") == 3.5
    assert b.whole_job_rate(1, 100, 50.0) == pytest.approx(2000.0)


def test_reference_arm_under_torchrun_prints_one_line():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"), "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    proc = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert proc.returncode == 0, proc.stderr[-2000:]
    lines = [ln for ln in proc.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
