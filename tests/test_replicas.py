"""The N > 1 bench path on CPU: two gloo ranks run the replica plumbing of
bench.py (per-rank inputs, timing barrier, max over ranks, whole-job rate)
and the reference arm, which only rank 0 runs."""
import contextlib
import io
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    from paper_1410_1599_gb300 import inputs as gen

    rep = bench.Replicas(rank, world, backend="gloo", device="cpu")
    rep.init()
    try:
        # every replica has its own inputs
        sa, sb = rep.seeds()
        A = gen.uniform_pm1(8, 8, 128, sa, -16, 16)
        B = gen.uniform_pm1(8, 8, 128, sb, -16, 16)
        digest = (sa, sb, int(A.limb.sum() % (1 << 61)), int(B.limb.sum() % (1 << 61)))
        seen = [None] * world
        dist.all_gather_object(seen, digest)
        assert len({d[:2] for d in seen}) == world
        assert len({d[2:] for d in seen}) == world
        # the step time is the slowest rank's; the rate counts every rank's work
        ms = [7.5, 11.25][rank]
        rep.barrier()
        slow = rep.allmax(ms)
        assert slow == 11.25
        assert rep.whole_job(1024.0, slow * 1e-3) == pytest.approx(world * 1024.0 / 11.25e-3)
        # reference arm: rank 0 times the oracle and prints one line; others do nothing
        ns = type("A", (), dict(n=24, prec=128, warmup=0, steps=1, algo="simple", cutoff=64))()
        out = io.StringIO()
        with contextlib.redirect_stdout(out):
            bench.run_reference(ns, rank, world)
        text = out.getvalue().strip()
        if rank == 0:
            line = json.loads(text)
            assert line["impl"] == "reference" and line["n_gpus"] == world
            assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
        else:
            assert text == ""
        rep.barrier()
    finally:
        rep.close()


def test_two_rank_replicas():
    import torch.multiprocessing as tmp
    tmp.spawn(_worker, args=(2, _free_port()), nprocs=2, join=True)


def test_single_rank_needs_no_process_group():
    import bench
    rep = bench.Replicas(0, 1, backend="gloo", device="cpu")
    rep.init()
    assert rep.allmax(3.5) == 3.5
    assert rep.whole_job(10.0, 2.0) == 5.0
    assert rep.seeds() == (3, 4)
    rep.barrier()
    rep.close()
