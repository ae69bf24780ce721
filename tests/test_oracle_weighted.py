"""Pins of the oracle's weighted averages over independent runs (Sec. VIII, Eqs.
weighted-averages and modified-weights2): hand-computed weights, invariances, the
fluctuating-size factor, and the log-normal closed form for the effective number of runs."""
import math

import numpy as np
import pytest

import oracle


def _obs(M, rng=None):
    rng = rng or np.random.default_rng(0)
    return rng.normal(size=(M, 5))


def test_two_runs_hand_computed():
    """-beta F differing by ln 2 at equal R: weights 1/3 and 2/3, M_eff = 1 / (1/9 + 4/9) =
    9/5, combined -beta F = ln((1 + 2) / 2)."""
    obs = np.array([[1, 2, 3, 4, 5], [4, 5, 6, 7, 8]], float)
    r = oracle.weighted_average([100, 100], [100, 100], [0.0, math.log(2)], [0, 0], obs, 1)
    assert r["e"] == pytest.approx(1 / 3 + 2 / 3 * 4, rel=1e-15)
    assert r["chi"] == pytest.approx(5 / 3 + 2 / 3 * 8, rel=1e-15)
    assert r["M_eff"] == pytest.approx(9 / 5, rel=1e-15) and r["max_weight"] == pytest.approx(2 / 3, rel=1e-15)
    assert r["minus_betaF_combined"] == pytest.approx(math.log(1.5), rel=1e-15)
    assert r["e_plain"] == 2.5 and r["var_minus_betaF"] == pytest.approx(math.log(2) ** 2 / 2, rel=1e-14)


def test_equal_runs_reduce_to_the_plain_mean():
    M = 7
    obs = _obs(M)
    r = oracle.weighted_average([500] * M, [500] * M, [-12.5] * M, [0.01] * M, obs, 1)
    assert r["M_eff"] == pytest.approx(M, rel=1e-14)
    for k, v in zip(["e", "C", "m", "m2", "chi"], obs.mean(axis=0)):
        assert r[k] == pytest.approx(v, rel=1e-13, abs=1e-15) and r[k + "_plain"] == pytest.approx(v, rel=1e-13, abs=1e-15)


def test_shift_invariance_and_mode_equivalence():
    """A common constant added to every -beta F changes no weight (it cancels in the
    normalisation) and shifts the combined free energy by itself; with all
    R_{k-1} = R (sum of ln(R_{k-1}/R) = 0) the two weightings coincide."""
    rng = np.random.default_rng(1)
    M = 12
    obs = _obs(M, rng)
    R_i = rng.integers(900, 1100, M).astype(float)
    mbF = rng.normal(-300, 0.7, M)
    a = oracle.weighted_average(R_i, [1000] * M, mbF, np.zeros(M), obs, 1)
    b = oracle.weighted_average(R_i, [1000] * M, mbF + 1234.5, np.zeros(M), obs, 1)
    c = oracle.weighted_average(R_i, [1000] * M, mbF, np.zeros(M), obs, 0)
    for k in ["e", "C", "m", "m2", "chi", "M_eff", "max_weight"]:
        assert a[k] == pytest.approx(b[k], rel=1e-12) and a[k] == pytest.approx(c[k], rel=1e-15)
    assert b["minus_betaF_combined"] - a["minus_betaF_combined"] == pytest.approx(1234.5, rel=1e-12)


def test_population_size_factors():
    """Eq. modified-weights2: a run whose past populations were larger by a factor e^s in
    total (sum of ln(R_{k-1}/R) = s) gets e^s times the weight; runs with equal free energy
    but different current sizes R_i are weighted in proportion to R_i (each replica counts
    once, Eq. weighted-averages)."""
    obs = np.array([[1, 0, 0, 0, 0], [0, 1, 0, 0, 0]], float)
    r = oracle.weighted_average([100, 100], [100, 100], [0.0, 0.0], [math.log(2), 0.0], obs, 1)
    assert r["e"] == pytest.approx(2 / 3, rel=1e-15) and r["C"] == pytest.approx(1 / 3, rel=1e-15)
    r0 = oracle.weighted_average([100, 100], [100, 100], [0.0, 0.0], [math.log(2), 0.0], obs, 0)
    assert r0["e"] == pytest.approx(0.5, rel=1e-15)
    r = oracle.weighted_average([300, 100], [300, 100], [0.0, 0.0], [0.0, 0.0], obs, 0)
    assert r["e"] == pytest.approx(0.75, rel=1e-15)


@pytest.mark.parametrize("sigma", [0.3, 0.7])
def test_lognormal_effective_number_of_runs(sigma):
    """-beta F ~ N(0, sigma^2) at equal R: the weights are log-normal, and
    M_eff / M = (sum w)^2 / (M sum w^2) -> E[w]^2 / E[w^2] = exp(-sigma^2) (Sec. VIII)."""
    rng = np.random.default_rng(7)
    M = 40000
    mbF = rng.normal(0.0, sigma, M)
    r = oracle.weighted_average(np.full(M, 1000.0), np.full(M, 1000.0), mbF, np.zeros(M), np.zeros((M, 5)), 1)
    assert r["M_eff"] / M == pytest.approx(math.exp(-sigma ** 2), rel=0.03)
    assert r["var_minus_betaF"] == pytest.approx(sigma ** 2, rel=0.03)


def test_multinomial_runs_have_no_size_factor():
    """Fixed-size (multinomial) resampling keeps R_{k-1} = R, so the size factor stays 0."""
    pa = oracle.PA(8, 400, 3, kind=oracle.MULTINOMIAL)
    pa.init()
    for i in range(1, 6):
        pa.resample(i / 10)
        pa.sweep(2)
    assert pa.observables()["sum_lnRratio"] == 0.0
    nr = oracle.PA(8, 400, 3)
    nr.init()
    for i in range(1, 6):
        nr.resample(i / 10)
        nr.sweep(2)
    assert nr.observables()["sum_lnRratio"] != 0.0
