"""One population split into P shards by contiguous slot ranges (pa_shard_*, Sec. II), all P
held on this GPU and exchanged through LocalTransport: at every step the concatenated spin
hashes, family ids and copy numbers, the combined histogram and every field of the step-4
record equal those of the same population held whole (pa_init / pa_resample /
pa_anneal_step), and the CPU oracle's."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402


def _whole(L, R, seed, kind, update):
    from paper_2102_06611_gb300 import PopulationAnnealing
    return PopulationAnnealing(L, R, seed, resample=kind, update=update)


def _sharded(L, R, seed, P, kind, update, capacity=None):
    from paper_2102_06611_gb300.shard import LocalTransport, ShardedRun, gpu_shards
    engines = gpu_shards(L, R, seed, list(range(P)), P, resample=kind, update=update, capacity=capacity)
    return ShardedRun(engines, P, LocalTransport()), engines


def _check_step(run, engines, whole, ref, with_counts):
    P = len(engines)
    obs = run.observables()
    want = whole.observables()
    assert obs == want, (obs, want)
    for e in engines.values():   # every shard holds the same whole-population record
        assert e.observables() == want
    assert np.array_equal(engines[0].histogram(), whole.histogram())
    hashes = np.concatenate([engines[s].hashes() for s in range(P)])
    assert np.array_equal(hashes, whole.hashes())
    fam = np.concatenate([engines[s].replicas()[2] for s in range(P)])
    assert np.array_equal(fam, whole.replicas()[2])
    if with_counts:
        counts = np.concatenate([engines[s].copy_counts() for s in range(P)])
        assert np.array_equal(counts, whole.copy_counts())
    if ref is not None:
        assert np.array_equal(hashes, ref.hashes())
        assert np.array_equal(fam, ref.state()[2])
        o = ref.observables()
        for k in ("e", "C", "m", "m2", "chi", "lnQ", "minus_betaF", "rho_t"):
            assert abs(obs[k] - o[k]) <= 1e-12 * max(1.0, abs(o[k])), (k, obs[k], o[k])
        assert obs["families"] == o["families"]
    bases = [engines[s].layout()[2] for s in range(P)]
    sizes = [engines[s].layout()[1] for s in range(P)]
    assert bases == [sum(sizes[:s]) for s in range(P)] and max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("L,R,P,kind,update,betas", [
    (16, 3001, 2, "nearest", "metropolis", [0.1, 0.2, 0.3, 0.45, 0.6]),
    (16, 3001, 3, "nearest", "metropolis", [0.1, 0.2, 0.3, 0.45, 0.6]),
    (10, 1999, 4, "poisson", "metropolis", [0.15, 0.3, 0.45, 0.6]),       # shared-memory sweep kernel
    (8, 777, 4, "nearest", "heatbath", [0.5, 1.0, 1.5, 2.0, 2.5, 3.0]),   # families span whole shards
    (32, 500, 1, "nearest", "metropolis", [0.2, 0.4]),                    # one shard
    (16, 2503, 3, "multinomial", "metropolis", [0.1, 0.25, 0.4, 0.6, 0.9]),
    (12, 1201, 4, "multinomial", "heatbath", [0.4, 0.9, 1.5, 2.2]),       # weights concentrated in few shards
])
def test_sharded_population_equals_whole(L, R, P, kind, update, betas):
    seed, theta = 9, 3
    run, engines = _sharded(L, R, seed, P, kind, update)
    whole = _whole(L, R, seed, kind, update)
    ref = oracle.PA(L, R, seed, kind={"nearest": oracle.NEAREST, "poisson": oracle.POISSON,
                                      "multinomial": oracle.MULTINOMIAL}[kind],
                    update=oracle.HEATBATH if update == "heatbath" else oracle.METROPOLIS)
    ref.init()
    _check_step(run, engines, whole, ref, False)
    for b in betas:
        run.resample(b)
        whole.resample(b)
        assert ref.resample(b) == 0
        run.anneal_step(theta)
        whole.anneal_step(theta)
        ref.sweep(theta)
        _check_step(run, engines, whole, ref, True)
    for e in engines.values():
        assert e.cur == e.layout()[0]
        e.close()
    whole.close()


@pytest.mark.parametrize("kind", ["nearest", "multinomial"])
def test_sharded_full_size_L64_R1e6(kind):
    """The headline population (L = 64, R = 10^6) in 4 shards: three temperature steps equal
    the whole population's, hash for hash."""
    L, R, P, seed, theta = 64, 1_000_000, 4, 7, 10
    run, engines = _sharded(L, R, seed, P, kind, "metropolis")
    whole = _whole(L, R, seed, kind, "metropolis")
    for i in (1, 2, 3):
        b = i / 300
        run.resample(b)
        whole.resample(b)
        run.anneal_step(theta)
        whole.anneal_step(theta)
        _check_step(run, engines, whole, None, True)
    for e in engines.values():
        e.close()
    whole.close()


def test_shard_call_order_is_enforced():
    """Out-of-order shard calls return PA_ERR_STATE and leave the context usable."""
    from paper_2102_06611_gb300 import PAError
    from paper_2102_06611_gb300.shard import gpu_shards
    e = gpu_shards(8, 100, 1, [0], 2)[0]
    with pytest.raises(PAError):
        e.resample(0.1)              # no combined histogram yet
    with pytest.raises(PAError):
        e.observables()              # likewise
    both = torch.stack([e.summary(), e.summary().clone()])   # two copies of shard 0: consistent
    e.combine(both)
    with pytest.raises(PAError):
        e.combine(both)              # once per measurement
    with pytest.raises(PAError):
        e.summary()                  # the histogram is already the combined one
    assert e.observables()["R"] == 100
    e.resample(0.1)
    with pytest.raises(PAError):
        e.anneal_step(1)             # the rebalanced population is not adopted yet
    n = min(e.local_size(), e.capacity)
    e.copy_children(0, n, e.views(0, n))
    e.adopt(n, 0)
    with pytest.raises(PAError):
        e.adopt(n, 0)                # once per resampling
    with pytest.raises(PAError):
        e.copy_children(0, 1, e.views(0, 1))   # likewise
    e.anneal_step(1)
    e.close()


def test_shard_combine_needs_its_own_row():
    """Summaries without a row of this shard's size at its slot base (e.g. not in slot order)
    set the sticky numeric error: the next synchronising call reports it."""
    from paper_2102_06611_gb300 import PAError
    from paper_2102_06611_gb300.shard import gpu_shards
    e = gpu_shards(8, 100, 1, [1], 2)[1]         # slots [50, 100)
    only = e.summary().unsqueeze(0)               # one row, starting at slot 0
    e.combine(only)
    with pytest.raises(PAError, match="NUMERIC"):
        e.observables()
    e.close()


def test_sharded_population_through_nccl_transport_one_rank():
    """The torch.distributed transport on this GPU: one NCCL rank holding 3 shards (summaries
    and children counts all-gathered by NCCL, children moved by direct copies), bit-identical
    to the whole population for a few steps."""
    import os
    import socket

    import torch.distributed as dist

    from paper_2102_06611_gb300.shard import DistTransport, ShardedRun, gpu_shards

    if dist.is_initialized():
        pytest.skip("a process group is already initialised")
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    os.environ.setdefault("NCCL_NVLS_ENABLE", "0")
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        L, R, seed, P, theta = 16, 2001, 5, 3, 3
        engines = gpu_shards(L, R, seed, list(range(P)), P)
        run = ShardedRun(engines, P, DistTransport(shards_per_rank=P))
        whole = _whole(L, R, seed, "nearest", "metropolis")
        _check_step(run, engines, whole, None, False)
        for b in (0.2, 0.4, 0.6):
            run.resample(b)
            whole.resample(b)
            run.anneal_step(theta)
            whole.anneal_step(theta)
            _check_step(run, engines, whole, None, True)
        for e in engines.values():
            e.close()
        whole.close()
    finally:
        dist.destroy_process_group()
