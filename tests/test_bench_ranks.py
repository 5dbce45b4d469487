"""The multi-rank (replicas) host logic of bench.py on CPU: two gloo ranks.

Each rank times its own replica; the job reports the slowest rank's time and
the units of all ranks (max over ranks, sum of units), and only rank 0 of the
reference arm prints.  No GPU is used."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        r, local, w = bench._dist()
        ms, units = bench.aggregate_ranks(10.0 + 5.0 * rank, 1000 * (rank + 1), "cpu", w)
        q.put((r, local, w, ms, units))
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_all_units():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[:3] for o in out] == [(0, 0, 2), (1, 1, 2)]
    for o in out:
        assert o[3] == 15.0 and o[4] == 3000.0


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(7.5, 42, "cpu", 1) == (7.5, 42.0)


def test_reference_arm_prints_on_rank_0_only():
    """Under torchrun with N > 1 the reference arm runs on rank 0 alone; the
    other ranks exit 0 without work or output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0 and r.stdout.strip() == ""
