"""Heatbath update (Sec. IV) on the GPU against the oracle, element by element: replica
hashes, level histograms, copy numbers and observables at every step, on the packed (L < 48)
and row-wise (L >= 48) sweep paths, at high and at low temperature (where most sites tie
with a threshold in their top 8 bits and the complemented low bits decide)."""
import numpy as np
import pytest

import oracle
from side_by_side import run_side_by_side

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pa(*a, **k):
    from paper_2102_06611_gb300 import PopulationAnnealing
    return PopulationAnnealing(*a, update="heatbath", **k)


def _ref(L, R, seed, kind="nearest", capacity=None):
    return oracle.PA(L, R, seed, kind=oracle.POISSON if kind == "poisson" else oracle.NEAREST, capacity=capacity,
                     update=oracle.HEATBATH)


RUNS = [
    # L, R, kind, betas, theta
    (4, 500, "nearest", [i / 10 for i in range(1, 11)], 3),
    (8, 1000, "nearest", [i / 20 for i in range(1, 21)], 5),
    (12, 300, "poisson", [0.2, 0.4, 0.6], 3),
    (16, 600, "nearest", [0.3, 0.6, 0.9], 3),
    (24, 300, "nearest", [0.3, 0.6, 1.0], 2),
    (32, 800, "poisson", [0.25, 0.5, 0.75, 1.0], 3),
    (48, 120, "nearest", [0.4, 0.8], 2),
    (64, 400, "nearest", [0.45, 0.7, 0.95], 3),
    (128, 150, "nearest", [0.5, 1.0], 2),
    (20, 300, "nearest", [0.3, 0.6, 1.0], 2),
    (40, 150, "poisson", [0.3, 0.6], 2),
    (80, 50, "nearest", [0.44, 0.9], 2),
    (96, 40, "nearest", [0.44, 1.0], 2),
]


@pytest.mark.parametrize("L,R,kind,betas,theta", RUNS)
def test_heatbath_run_parity(L, R, kind, betas, theta):
    gpu = _pa(L, R, seed=4, resample=kind)
    ref = _ref(L, R, 4, kind, capacity=gpu.capacity)
    run_side_by_side(gpu, ref, betas, theta)


@pytest.mark.parametrize("L", [4, 8, 16, 32, 64, 128])
def test_heatbath_at_beta_zero(L):
    """At beta = 0 a site flips iff the top bit of its uniform is 0 (probability 1/2): the
    sweep matches the oracle and flips about half of the spins."""
    gpu = _pa(L, 64, seed=9)
    ref = _ref(L, 64, 9, capacity=gpu.capacity)
    ref.init()
    before = gpu.export_spins()
    gpu.anneal_step(1)
    ref.sweep(1)
    assert np.array_equal(gpu.hashes(), ref.hashes())
    after = gpu.export_spins()
    flipped = sum(bin(int(x)).count("1") for x in np.bitwise_xor(before, after).reshape(-1))
    assert 0.4 < flipped / (64 * L * L) < 0.6


def test_heatbath_split_sweeps_and_checkpoint():
    """Sweeps split over calls equal one call, and a checkpoint taken between them resumes
    bit for bit (the update kind is part of the configuration)."""
    a = _pa(32, 500, seed=2)
    b = _pa(32, 500, seed=2)
    a.resample(0.4)
    b.resample(0.4)
    a.anneal_step(5)
    b.anneal_step(2)
    ck = b.save()
    c = _pa(32, 500, seed=2)
    c.load(ck)
    b.anneal_step(3)
    c.anneal_step(3)
    assert np.array_equal(a.hashes(), b.hashes()) and np.array_equal(a.hashes(), c.hashes())
    from paper_2102_06611_gb300 import PAError, PopulationAnnealing
    m = PopulationAnnealing(32, 500, 2)   # Metropolis: a different configuration
    with pytest.raises(PAError):
        m.load(ck)


def test_heatbath_differs_from_metropolis():
    from paper_2102_06611_gb300 import PopulationAnnealing
    h = _pa(16, 200, seed=1)
    m = PopulationAnnealing(16, 200, 1)
    for pa in (h, m):
        pa.resample(0.3)
        pa.anneal_step(2)
    assert not np.array_equal(h.hashes(), m.hashes())
