"""Lattice sizes without a register kernel (any even 4 <= L <= 128 other than 4, 8, 12, 16,
20, 24, 32, 40, 48, 64, 80, 96, 128) run the shared-memory sweep kernel; they follow the same definitions
(Sec. II step list, Sec. IV updates), so the GPU matches the oracle element by element:
spin hashes, histograms, copy numbers, levels, magnetisations, family ids and observables at
every step, for both updates and all three resampling kinds, on sizes whose rows span a
fraction of a 32-site chunk (L < 34), one chunk (34 <= L <= 64) or two (L > 64)."""
import numpy as np
import pytest

import oracle
from side_by_side import compare_population, run_side_by_side

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KIND = {"nearest": oracle.NEAREST, "poisson": oracle.POISSON, "multinomial": oracle.MULTINOMIAL}


def _pair(L, R, seed, kind="nearest", update="metropolis"):
    from paper_2102_06611_gb300 import PopulationAnnealing
    gpu = PopulationAnnealing(L, R, seed, resample=kind, update=update)
    ref = oracle.PA(L, R, seed, kind=KIND[kind], capacity=gpu.capacity,
                    update=oracle.HEATBATH if update == "heatbath" else oracle.METROPOLIS)
    return gpu, ref


RUNS = [
    # L, R, kind, update, betas, theta
    (6, 400, "nearest", "metropolis", [i / 10 for i in range(1, 11)], 3),
    (10, 300, "poisson", "metropolis", [0.2, 0.4, 0.6, 0.8], 3),
    (14, 300, "nearest", "heatbath", [0.25, 0.5, 0.75], 2),
    (18, 250, "multinomial", "metropolis", [0.3, 0.44, 0.6], 3),
    (22, 200, "nearest", "metropolis", [0.4, 0.9], 2),
    (34, 150, "nearest", "metropolis", [0.3, 0.44, 1.0], 2),
    (42, 150, "poisson", "heatbath", [0.3, 0.6], 2),
    (50, 100, "nearest", "metropolis", [0.44, 0.8], 2),
    (66, 60, "nearest", "metropolis", [0.35, 0.7], 2),
    (94, 40, "nearest", "heatbath", [0.44, 1.0], 2),
    (100, 40, "poisson", "metropolis", [0.5, 1.0], 2),
    (126, 30, "nearest", "metropolis", [0.44, 0.9], 1),
]


@pytest.mark.parametrize("L,R,kind,update,betas,theta", RUNS)
def test_any_L_run_parity(L, R, kind, update, betas, theta):
    gpu, ref = _pair(L, R, 3, kind, update)
    run_side_by_side(gpu, ref, betas, theta)


@pytest.mark.parametrize("L", [6, 18, 30, 36, 62, 70, 126])
def test_any_L_beta_zero_flips_every_site(L):
    """At beta = 0 every Metropolis threshold is 2^32: one sweep flips every site (both
    colours), so the population after it is the complement of the initial one."""
    from paper_2102_06611_gb300 import PopulationAnnealing
    gpu = PopulationAnnealing(L, 50, seed=2)
    ref = oracle.PA(L, 50, 2, capacity=gpu.capacity)
    ref.init()
    compare_population(gpu, ref, "init")
    before = gpu.export_spins()
    gpu.anneal_step(1)
    ref.sweep(1)
    compare_population(gpu, ref, "after one sweep at beta = 0")
    after = gpu.export_spins()
    mask = np.zeros_like(before)
    words = (L + 31) // 32
    for w in range(words):
        bits = min(32, L - 32 * w)
        mask.reshape(-1, L, words)[:, :, w] = (1 << bits) - 1 if bits < 32 else 0xFFFFFFFF
    assert np.array_equal(after, before ^ mask)


def test_any_L_split_sweeps_and_checkpoint():
    """Sweeps split over calls equal one call (sweep numbering continues within the step),
    and a checkpoint taken between them resumes bit for bit."""
    from paper_2102_06611_gb300 import PopulationAnnealing
    a = PopulationAnnealing(42, 300, 5)
    b = PopulationAnnealing(42, 300, 5)
    for pa in (a, b):
        pa.resample(0.4)
    a.anneal_step(5)
    b.anneal_step(2)
    ck = b.save()
    c = PopulationAnnealing(42, 300, 5)
    c.load(ck)
    b.anneal_step(3)
    c.anneal_step(3)
    assert np.array_equal(a.hashes(), b.hashes()) and np.array_equal(a.hashes(), c.hashes())
    assert np.array_equal(a.histogram(), c.histogram())


def test_any_L_larger_population_sampled():
    """L = 100, R = 20000 (several blocks of the grid, every warp with many replicas): the
    oracle sweeps a sample of the GPU's own replicas after resampling and must reproduce their
    spins; the histogram of the whole population matches the GPU's levels."""
    from paper_2102_06611_gb300 import PopulationAnnealing
    L, R = 100, 20000
    gpu = PopulationAnnealing(L, R, 11)
    gpu.resample(0.3)
    words0 = gpu.export_spins()
    gpu.anneal_step(2)
    words1 = gpu.export_spins()
    rng = np.random.default_rng(0)
    for j in rng.choice(gpu.R, 12, replace=False):
        s0 = oracle.unpack(L, words0[j].reshape(-1))
        s1 = oracle.sweep_replica(L, 11, 1, int(j), 0.3, 2, s0)
        assert np.array_equal(oracle.pack(L, s1), words1[j].reshape(-1)), f"replica {j}"
    lv, _, _ = gpu.replicas()
    assert np.array_equal(np.bincount(lv, minlength=L * L + 1), gpu.histogram())

