"""The sharded single run (one population split over ranks by contiguous slot ranges,
paper_2102_06611_gb300.shard) on gloo ranks, CPU only, with the oracle-based shard engine of
tests/shard_oracle.py: at every step the spin hashes, copy numbers, family ids, the whole
population's histogram and the observables must equal those of the oracle's one population
(Sec. II), for 2 and 4 ranks, uneven shard sizes, 2 shards per rank, nearest-integer and
Poisson resampling, and a schedule harsh enough that families span whole shards."""
import os
import socket
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402

FIELDS = [f for f in oracle.OBS_FIELDS]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, outdir, L, R, seed, kind, betas, theta, per_rank, update):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    import pickle

    import torch.distributed as dist

    from paper_2102_06611_gb300.shard import DistTransport, ShardedRun, shard_capacity, split
    from shard_oracle import OracleShard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    P = world * per_rank
    cap = shard_capacity(R, P)
    engines = {}
    for s in range(rank * per_rank, (rank + 1) * per_rank):
        lo, hi = split(R, P, s)
        engines[s] = OracleShard(L, R, seed, lo, hi - lo, cap, kind=kind, update=update)
    run = ShardedRun(engines, P, DistTransport(shards_per_rank=per_rank))
    log = []

    def snap():
        rec = {"obs": run.observables(), "hist": next(iter(engines.values())).glob["hist"].copy(), "shards": {}}
        for s, e in engines.items():
            rec["shards"][s] = {"hashes": e.hashes(), "fam": e.families(), "counts": e.counts.copy(),
                                "base": e.base}
        log.append(rec)

    snap()
    for b in betas:
        run.resample(b)
        run.anneal_step(theta)
        snap()
    with open(os.path.join(outdir, f"rank{rank}.pkl"), "wb") as f:
        pickle.dump(log, f)
    dist.barrier()
    dist.destroy_process_group()


def _reference(L, R, seed, kind, betas, theta, update=oracle.METROPOLIS):
    pa = oracle.PA(L, R, seed, kind=kind, update=update)
    pa.init()
    out = []

    def snap(counts):
        o = pa.observables()
        out.append({"obs": {k: o[k] for k in FIELDS}, "hist": pa.histogram().astype(np.int64),
                    "hashes": pa.hashes(), "fam": pa.state()[2], "counts": counts})

    snap(np.zeros(0, np.int32))
    for b in betas:
        assert pa.resample(b) == 0
        counts = pa.counts()
        pa.sweep(theta)
        snap(counts)
    return out


def _run_sharded(world, per_rank, L, R, seed, kind, betas, theta, update=oracle.METROPOLIS):
    import pickle

    import torch.multiprocessing as mp
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main, args=(world, _free_port(), d, L, R, seed, kind, betas, theta, per_rank, update),
                           nprocs=world, join=True, start_method="spawn")
        logs = [pickle.load(open(os.path.join(d, f"rank{r}.pkl"), "rb")) for r in range(world)]
    return logs


def _compare(logs, ref):
    for i, want in enumerate(ref):
        shards = {}
        for log in logs:
            shards.update(log[i]["shards"])
            assert log[i]["obs"] == {k: want["obs"][k] for k in FIELDS}, (i, log[i]["obs"], want["obs"])
            assert np.array_equal(log[i]["hist"], want["hist"]), i
        order = sorted(shards)
        bases = [shards[s]["base"] for s in order]
        assert bases == sorted(bases)
        assert np.array_equal(np.concatenate([shards[s]["hashes"] for s in order]), want["hashes"]), i
        assert np.array_equal(np.concatenate([shards[s]["fam"] for s in order]), want["fam"]), i
        if i > 0:
            assert np.array_equal(np.concatenate([shards[s]["counts"] for s in order]), want["counts"]), i


@pytest.mark.parametrize("world,per_rank,R,kind,betas,update", [
    (2, 1, 301, oracle.NEAREST, [0.1, 0.25, 0.4, 0.55, 0.7], oracle.METROPOLIS),
    (4, 1, 257, oracle.POISSON, [0.15, 0.3, 0.45, 0.6], oracle.METROPOLIS),
    (2, 2, 203, oracle.NEAREST, [0.5, 1.0, 1.5, 2.0, 2.5], oracle.METROPOLIS),   # harsh: families span shards
    (2, 2, 211, oracle.MULTINOMIAL, [0.1, 0.3, 0.6, 1.0, 1.6], oracle.METROPOLIS),
    (2, 1, 233, oracle.POISSON, [0.2, 0.4, 0.7, 1.0], oracle.HEATBATH),
])
def test_sharded_run_matches_one_population(world, per_rank, R, kind, betas, update):
    L, seed, theta = 8, 11, 2
    ref = _reference(L, R, seed, kind, betas, theta, update)
    logs = _run_sharded(world, per_rank, L, R, seed, kind, betas, theta, update)
    _compare(logs, ref)
    if betas[-1] >= 2.0:  # the harsh schedule did collapse the families below the shard count
        assert ref[-1]["obs"]["families"] < world * per_rank


def test_rebalance_plan():
    """The re-split: children of shard s occupy [o_s, o_s + c_s) (o = exclusive scan), new
    ranges are even, every replica moves exactly once."""
    from paper_2102_06611_gb300.shard import rebalance_plan, split
    rng = np.random.default_rng(4)
    for P in (1, 2, 3, 4, 7):
        for _ in range(50):
            totals = [int(x) for x in rng.integers(0, 40, P)]
            if sum(totals) == 0:
                continue
            plan = rebalance_plan(totals)
            R = sum(totals)
            assert plan.R_total == R and sum(plan.size) == R
            assert [plan.lo[t] for t in range(P)] == [split(R, P, t)[0] for t in range(P)]
            offs = np.concatenate([[0], np.cumsum(totals)])
            seen = np.zeros(R, int)
            for tr in plan.transfers:
                g0 = offs[tr.src] + tr.src_off
                assert g0 == plan.lo[tr.dst] + tr.dst_off
                assert 0 <= tr.src_off and tr.src_off + tr.count <= totals[tr.src]
                assert 0 <= tr.dst_off and tr.dst_off + tr.count <= plan.size[tr.dst]
                seen[g0:g0 + tr.count] += 1
            assert np.all(seen == 1)
    plan = rebalance_plan([5, 5])
    assert [(t.src, t.src_off, t.dst, t.dst_off, t.count) for t in plan.transfers] == [(0, 0, 0, 0, 5), (1, 0, 1, 0, 5)]
    plan = rebalance_plan([9, 0, 3])
    assert plan.size == [4, 4, 4]
    assert [(t.src, t.src_off, t.dst, t.dst_off, t.count) for t in plan.transfers] == \
        [(0, 0, 0, 0, 4), (0, 4, 1, 0, 4), (0, 8, 2, 0, 1), (2, 0, 2, 1, 3)]
