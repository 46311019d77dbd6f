"""The multi-rank path of bench.py on the CPU: two gloo ranks (127.0.0.1) take every timing's
maximum over the ranks, and the reference arm runs on rank 0 alone."""
import argparse
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank-dependent timings: the slowest replica must set every entry
        vals = bench.max_over_ranks([10.0 + rank, 5.0 - rank, 0.5 * rank, 7.0], world)
        torch.distributed.barrier()
        q.put((rank, vals))
    finally:
        torch.distributed.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    try:
        for _ in range(2):
            rank, vals = q.get(timeout=120)
            got[rank] = vals
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    assert got[0] == got[1] == [11.0, 5.0, 0.5, 7.0]


def test_max_over_ranks_single_rank_is_identity():
    assert bench.max_over_ranks([3.0, 1.5], 1) == [3.0, 1.5]


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the ranks other than 0 leave the reference arm without any work."""
    args = argparse.Namespace(steps=1, warmup=1, cpu_scale=8)
    assert bench.run_reference(args, 1, 2) is None
