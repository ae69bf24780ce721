"""Fixed-size multinomial resampling (Sec. II) on the GPU against the oracle: copy numbers,
replica hashes, histograms and observables at every step, R_i = R throughout, and a
full-size replay of the copy numbers from the device's own levels."""
import numpy as np
import pytest

import oracle
from side_by_side import run_side_by_side

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pa(*a, **k):
    from paper_2102_06611_gb300 import PopulationAnnealing
    return PopulationAnnealing(*a, resample="multinomial", **k)


@pytest.mark.parametrize("L,R,nT,theta,update", [
    (4, 700, 21, 3, "metropolis"),
    (8, 1000, 51, 5, "metropolis"),
    (16, 2500, 11, 3, "heatbath"),
    (32, 1025, 9, 2, "metropolis"),
    (64, 300, 5, 2, "metropolis"),
])
def test_multinomial_run_parity(L, R, nT, theta, update):
    gpu = _pa(L, R, seed=6, update=update)
    ref = oracle.PA(L, R, 6, kind=oracle.MULTINOMIAL, capacity=gpu.capacity,
                    update=oracle.HEATBATH if update == "heatbath" else oracle.METROPOLIS)
    run_side_by_side(gpu, ref, [i / (nT - 1) for i in range(1, nT)], theta)
    assert gpu.R == R


def test_multinomial_full_size_copy_numbers():
    """L = 32, R = 10^5: the oracle recomputes every copy number from the device's levels
    before each of three resamplings (beta = 0.3, 0.6, 0.9 after theta = 5 sweeps each)."""
    L, R, seed = 32, 100_000, 3
    gpu = _pa(L, R, seed=seed)
    beta_prev = 0.0
    for i, beta in enumerate((0.3, 0.6, 0.9), start=1):
        lv, _, fm = gpu.replicas()
        gpu.resample(beta)
        st, counts, lnQ, S, kmin, R_new = oracle.resample_levels(L, R, lv, beta_prev, beta, i, seed,
                                                                 oracle.MULTINOMIAL, gpu.capacity)
        assert st == 0 and R_new == R
        assert np.array_equal(gpu.copy_counts(), counts), f"step {i}"
        assert gpu.R == R
        lv2, _, fm2 = gpu.replicas()
        parents = np.repeat(np.arange(len(lv)), counts)
        assert np.array_equal(lv2, lv[parents]) and np.array_equal(fm2, fm[parents])
        gpu.anneal_step(5)
        obs = gpu.observables()
        assert abs(obs["lnQ"] - lnQ) <= 1e-12 * max(1.0, abs(lnQ))
        beta_prev = beta
