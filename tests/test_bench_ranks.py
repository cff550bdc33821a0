"""Host logic of bench.py's multi-GPU mode on CPU (gloo, world size 2).

Under torchrun every rank runs an independent replica; the step time that
enters the reported throughput is the largest over the ranks, and only rank 0
runs the oracle reference arm.  These tests run that logic with the gloo
backend in two spawned processes, without a GPU.
"""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=2)
    try:
        import bench
        q.put((rank, bench.max_over_ranks(1.5 + rank, 2, "cpu"), bench.max_over_ranks(7.0 - rank, 2, "cpu")))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_gloo():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(out) == [(0, 2.5, 7.0), (1, 2.5, 7.0)]


def test_single_rank_max_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1, "cpu") == 3.25


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        workload = "many_disks"
        steps = 1
        warmup = 3

    assert bench.run_reference(Args(), 2, 1) is None
    assert capsys.readouterr().out == ""
