"""Batches vs single runs: every run of a mixed batch (different L, R, temperatures, theta,
seed, resampling) must end bit-identical to a single-run context driven with the same
linear schedule, and one failing run must not disturb the others."""
import numpy as np
import pytest

import oracle
from side_by_side import assert_obs_close, compare_population

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _single(spec):
    from paper_2102_06611_gb300 import PopulationAnnealing
    pa = PopulationAnnealing(spec.L, spec.R, spec.seed, resample=spec.resample, capacity=spec.capacity,
                             update=spec.update)
    for i in range(1, spec.n_temps):
        pa.resample(i / (spec.n_temps - 1))
        pa.anneal_step(spec.theta)
    return pa


MIXED = [
    # L, R, seed, n_temps, theta, resample
    (64, 700, 11, 6, 3, "nearest"),
    (8, 2000, 12, 11, 1, "nearest"),
    (12, 500, 13, 4, 5, "poisson"),
    (16, 1200, 14, 9, 0, "nearest"),
    (24, 300, 15, 7, 2, "nearest"),
    (32, 900, 16, 5, 4, "poisson"),
    (48, 150, 17, 3, 2, "nearest"),
    (4, 3000, 18, 12, 3, "nearest"),
    (128, 20, 19, 3, 1, "nearest"),
]


@pytest.mark.parametrize("shape", [None, (1, 2, 1), (0, 1, 2), (1, 1, 4)])
def test_mixed_batch_matches_single_runs(shape):
    """The autotuner's shape, and fixed shapes: one launch over every size or one per size,
    1-2 blocks per SM, 1-4x the default replica groups per work item."""
    from paper_2102_06611_gb300.batch import Batch, RunSpec
    specs = [RunSpec(L, R, seed, nT, th, kind) for (L, R, seed, nT, th, kind) in MIXED]
    b = Batch(specs)
    if shape is not None:
        b.set_shape(*shape)
        assert b.tuning()["chosen"] is None
    steps = b.run_to_end()
    assert steps == max(s.n_temps for s in specs) - 1
    active, status, step = b.status()
    assert not active.any() and not status.any()
    assert list(step) == [s.n_temps - 1 for s in specs]
    recs = b.observables()
    for i, s in enumerate(specs):
        pa = _single(s)
        assert np.array_equal(b.hashes(i), pa.hashes()), i
        o = pa.observables()
        for k in ("step", "R", "beta", "dbeta", "e", "C", "m", "m2", "chi", "lnQ", "minus_betaF", "rho_t",
                  "families", "sum_E", "sum_E2", "sum_absM", "sum_M2", "sum_size2", "theta"):
            assert recs[i][k] == o[k], (i, k, recs[i][k], o[k])
        pa.close()
    t = b.tuning()
    if shape is None:
        # the fastest shape, or the fastest single launch within 2 % of it
        fastest = min(c["ms"] for c in t["candidates"])
        best_one = min(c["ms"] for c in t["candidates"] if c["unified"])
        assert t["chosen"] in t["candidates"]
        if best_one <= 1.02 * fastest:
            assert t["chosen"]["unified"] == 1 and t["chosen"]["ms"] == best_one
        else:
            assert t["chosen"]["ms"] == fastest
        assert {c["unified"] for c in t["candidates"]} == {0, 1}


HEATBATH_MIX = [
    # L, R, seed, n_temps, theta, resample, update
    (64, 500, 31, 6, 3, "nearest", "heatbath"),
    (64, 600, 32, 5, 2, "multinomial", "metropolis"),
    (16, 1500, 33, 8, 4, "poisson", "heatbath"),
    (32, 700, 34, 7, 1, "nearest", "heatbath"),
    (8, 900, 35, 9, 5, "multinomial", "metropolis"),
    (128, 30, 36, 4, 2, "nearest", "heatbath"),
    (12, 800, 37, 5, 3, "multinomial", "heatbath"),
    (24, 2500, 38, 6, 2, "nearest", "metropolis"),
]


@pytest.mark.parametrize("shape", [None, (1, 1, 1)])
def test_batch_with_heatbath_and_multinomial_runs_matches_single_runs(shape):
    """Heatbath (Sec. IV) and Metropolis runs, with nearest-integer, Poisson and fixed-size
    multinomial resampling (Sec. II), in one batch: each bit-identical to its single run, with
    the per-size launches and with the launch over every size."""
    from paper_2102_06611_gb300.batch import Batch, RunSpec
    specs = [RunSpec(L, R, seed, nT, th, kind, update=u) for (L, R, seed, nT, th, kind, u) in HEATBATH_MIX]
    b = Batch(specs)
    if shape is not None:
        b.set_shape(*shape)
    b.run_to_end()
    active, status, step = b.status()
    assert not active.any() and not status.any()
    recs = b.observables()
    for i, s in enumerate(specs):
        pa = _single(s)
        assert np.array_equal(b.hashes(i), pa.hashes()), i
        o = pa.observables()
        for k in ("step", "R", "lnQ", "minus_betaF", "sum_E", "sum_E2", "sum_absM", "sum_M2", "families"):
            assert recs[i][k] == o[k], (i, k, recs[i][k], o[k])
        pa.close()
    b.close()


def test_batch_run_against_oracle():
    from paper_2102_06611_gb300.batch import Batch, RunSpec
    spec = RunSpec(8, 600, 5, 9, 3)
    b = Batch([spec, RunSpec(16, 400, 6, 5, 2)])
    ref = oracle.PA(8, 600, 5, capacity=spec.capacity or None)
    ref.init()
    for i in range(1, 9):
        b.step()
        assert ref.resample(i / 8) == 0
        ref.sweep(3)
    assert np.array_equal(b.hashes(0), ref.hashes())
    assert_obs_close(b.observables()[0], ref.observables(), "batched run 0")


def test_failing_run_is_isolated():
    from paper_2102_06611_gb300.batch import Batch, RunSpec
    good = RunSpec(16, 800, 21, 8, 2)
    bad = RunSpec(4, 500, 22, 40, 1, "poisson", capacity=500)  # the population outgrows its capacity
    b = Batch([bad, good])
    b.run_to_end()
    active, status, step = b.status()
    assert status[0] == 3 and status[1] == 0 and step[1] == 7
    pa = _single(good)
    assert np.array_equal(b.hashes(1), pa.hashes())


def test_full_mixed_batch_first_steps_match_single_runs():
    """The 64-run mixed workload at full size (L in {8, ..., 64}, R up to 2e5, theta in {1, 5,
    10}): after three batched temperature steps every run is bit-identical to its single run
    (spin hashes and records)."""
    from paper_2102_06611_gb300 import PopulationAnnealing
    from paper_2102_06611_gb300.batch import Batch, mixed_runs
    specs = mixed_runs()
    b = Batch(specs)
    k = 3
    for _ in range(k):
        b.step()
    recs = b.observables()
    for i, s in enumerate(specs):
        pa = PopulationAnnealing(s.L, s.R, s.seed, resample=s.resample, capacity=s.capacity)
        for j in range(1, k + 1):
            pa.resample(j / (s.n_temps - 1))
            pa.anneal_step(s.theta)
        assert np.array_equal(b.hashes(i), pa.hashes()), i
        o = pa.observables()
        for key in ("step", "R", "beta", "lnQ", "minus_betaF", "sum_E", "sum_E2", "sum_absM", "sum_M2", "families"):
            assert recs[i][key] == o[key], (i, key)
        pa.close()
    b.close()


def test_full_mixed_batch_runs_against_oracle():
    """The 64-run mixed workload at full size: after three batched temperature steps, eight of
    its runs (every lattice size present but 64, small enough to replay) agree with the CPU
    oracle's own runs -- spin hashes bit for bit, observables to 1e-12."""
    from paper_2102_06611_gb300.batch import Batch, mixed_runs
    specs = mixed_runs()
    b = Batch(specs)
    k = 3
    for _ in range(k):
        b.step()
    recs = b.observables()
    for i in (0, 2, 7, 14, 27, 40, 46, 63):
        s = specs[i]
        ref = oracle.PA(s.L, s.R, s.seed)
        ref.init()
        for j in range(1, k + 1):
            assert ref.resample(j / (s.n_temps - 1)) == 0
            ref.sweep(s.theta)
        assert np.array_equal(b.hashes(i), ref.hashes()), (i, s)
        assert_obs_close(recs[i], ref.observables(), f"run {i}")
    b.close()


ANY_L_MIX = [
    # L, R, seed, n_temps, theta, resample, update: sizes without a register sweep kernel
    (6, 3000, 41, 7, 3, "nearest", "metropolis"),
    (10, 1200, 42, 6, 2, "poisson", "heatbath"),
    (20, 900, 43, 5, 4, "nearest", "metropolis"),
    (40, 400, 44, 6, 1, "multinomial", "metropolis"),
    (100, 60, 45, 4, 2, "nearest", "heatbath"),
    (64, 500, 46, 5, 2, "nearest", "metropolis"),
    (16, 800, 47, 8, 3, "nearest", "metropolis"),
]


@pytest.mark.parametrize("shape", [None, (1, 1, 1)])
def test_batch_with_every_even_L_matches_single_runs(shape):
    """Runs of even L without a batched register kernel (the shared-memory sweep, batched)
    beside register sizes in one batch, each bit-identical to its single run (which, at L =
    20 and 40, runs the single-run register kernel: two kernels, one result)."""
    from paper_2102_06611_gb300.batch import Batch, RunSpec
    specs = [RunSpec(L, R, seed, nT, th, kind, update=u) for (L, R, seed, nT, th, kind, u) in ANY_L_MIX]
    b = Batch(specs)
    if shape is not None:
        b.set_shape(*shape)
    b.run_to_end()
    active, status, step = b.status()
    assert not active.any() and not status.any()
    recs = b.observables()
    for i, s in enumerate(specs):
        pa = _single(s)
        assert np.array_equal(b.hashes(i), pa.hashes()), i
        o = pa.observables()
        for k in ("step", "R", "lnQ", "minus_betaF", "sum_E", "sum_E2", "sum_absM", "sum_M2", "families", "theta"):
            assert recs[i][k] == o[k], (i, k, recs[i][k], o[k])
        pa.close()
    b.close()
