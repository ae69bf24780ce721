"""The several-GPU path on CPU ranks: world size 2 over gloo.  Ranks run independent
populations (seed + rank) and the measurement takes the slowest rank's time and the sum of
the work; the oracle stands in for each rank's population."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2102_06611_gb300.multi import aggregate, rank_seed
        pa = oracle.PA(8, 300, rank_seed(7, rank))
        pa.init()
        attempts = 0
        for i in range(1, 4):
            pa.resample(i / 10)
            pa.sweep(2)
            attempts += 64 * pa.R * 2
        ms = 10.0 + 5.0 * rank
        res = aggregate(ms, ms / 2, attempts)
        h = pa.hashes()
        out[rank] = (res, int(h[0]), attempts)
    finally:
        dist.destroy_process_group()


def test_two_ranks_aggregate_and_differ():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True,
                           start_method="spawn")
        r0, r1 = out[0], out[1]
    assert r0[0] == r1[0]                       # every rank sees the same aggregate
    ms, sweep_ms, attempts = r0[0]
    assert ms == 15.0 and sweep_ms == 7.5       # the slowest rank
    assert attempts == r0[2] + r1[2]            # total work of both populations
    assert r0[1] != r1[1]                       # independent populations (seed + rank)


def test_single_process_aggregate_is_identity():
    from paper_2102_06611_gb300.multi import aggregate
    assert aggregate(3.0, 1.0, 42.0) == (3.0, 1.0, 42.0)
