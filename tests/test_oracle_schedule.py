"""Pins of the oracle's adaptive-schedule pieces: the energy-histogram overlap alpha and the
bisection on the temperature step (Sec. II, Sec. V's overlap kappa_i, Sec. VIII's alpha,
and the alpha > 0.7 guideline of Sec. X)."""
import math

import numpy as np
import pytest

import oracle


def _boltzmann_hist(g, beta, scale=1e15):
    N = len(g) - 1
    E = 4 * np.arange(N + 1) - 2 * N
    w = g * np.exp(-beta * (E - E.min()))
    return np.rint(w / w.sum() * scale).astype(np.int64)


def test_overlap_at_zero_step_is_one():
    g, _, _ = oracle.bruteforce(4)
    assert oracle.overlap(16, g, 0.0) == 1.0
    assert oracle.overlap(16, _boltzmann_hist(g, 0.4), 0.0) == pytest.approx(1.0, abs=1e-15)


@pytest.mark.parametrize("beta,dbeta", [(0.0, 0.05), (0.3, 0.1), (0.44, 0.2), (0.7, 0.5)])
def test_overlap_equals_exact_distribution_overlap_L4(beta, dbeta):
    """With a histogram proportional to the exact Boltzmann distribution at beta (L=4,
    enumeration), alpha(dbeta) is the overlap of the exact distributions at beta and
    beta + dbeta."""
    g, _, _ = oracle.bruteforce(4)
    E = 4 * np.arange(17) - 32

    def P(b):
        w = g * np.exp(-b * (E - E.min()))
        return w / w.sum()

    exact = float(np.minimum(P(beta), P(beta + dbeta)).sum())
    assert oracle.overlap(16, _boltzmann_hist(g, beta), dbeta) == pytest.approx(exact, abs=1e-9)


def _gauss_hist(N, mean_E, sigma, scale=1e12):
    E = 4 * np.arange(N + 1) - 2 * N
    w = np.exp(-0.5 * ((E - mean_E) / sigma) ** 2)
    return np.rint(w / w.sum() * scale).astype(np.int64)


def test_overlap_gaussian_closed_form():
    """For a Gaussian energy distribution of width sigma, reweighting shifts the mean by
    -dbeta sigma^2 and alpha = 2 Phi(-dbeta sigma / 2) = erfc(dbeta sigma / (2 sqrt 2))."""
    L = 64
    N = L * L
    sigma = math.sqrt(2 * N)  # the beta = 0 width, sigma_0^2 = 2N (Sec. VIII)
    h = _gauss_hist(N, 0.0, sigma)
    for db in (0.005, 0.01, 0.02, 0.04):
        expect = math.erfc(db * sigma / (2 * math.sqrt(2)))
        assert oracle.overlap(N, h, db) == pytest.approx(expect, abs=3e-3)


def test_overlap_matches_the_papers_numbers_at_criticality_L32():
    """Sec. VIII: for L = 32 at beta_c the overlap is about 0.3 at dbeta = 0.02 and below 10 %
    for dbeta >= 0.05.  The energy width at beta_c comes from the exact specific heat."""
    L = 32
    N = L * L
    bc = 0.5 * math.log(1 + math.sqrt(2))
    e_mean, C, _ = oracle.kaufman_thermo(L, bc)
    sigma = math.sqrt(C * N) / bc
    h = _gauss_hist(N, e_mean, sigma)
    assert abs(oracle.overlap(N, h, 0.02) - 0.3) < 0.05
    assert oracle.overlap(N, h, 0.05) < 0.10


def test_overlap_decreases_with_step():
    pa = oracle.PA(16, 4000, seed=2)
    pa.init()
    pa.resample(0.3)
    pa.sweep(5)
    h = pa.histogram().astype(np.int64)
    a = [oracle.overlap(256, h, db) for db in np.linspace(0.0, 0.3, 61)]
    assert all(x >= y for x, y in zip(a, a[1:]))


@pytest.mark.parametrize("target", [0.5, 0.8, 0.95])
def test_bisection_finds_the_largest_step_reaching_the_target(target):
    pa = oracle.PA(16, 4000, seed=3)
    pa.init()
    pa.resample(0.2)
    pa.sweep(5)
    h = pa.histogram().astype(np.int64)
    N = 256
    b_next, a = oracle.bisect_next_beta(N, h, 0.2, 1.0, 0.1, target)
    db = b_next - 0.2
    assert 0 < db <= 0.1
    # (db here is (beta + dbeta) - beta, within an ulp of the bisection's dbeta)
    assert a >= target and a == pytest.approx(oracle.overlap(N, h, db), abs=1e-12)
    if db < 0.1 - 1e-15:
        # a slightly larger step misses the target (1e-9 moves alpha far more than its
        # rounding noise of ~1e-15)
        assert oracle.overlap(N, h, db + 1e-9) < target


def test_bisection_end_of_schedule():
    g, _, _ = oracle.bruteforce(4)
    h = _boltzmann_hist(g, 0.95)
    b, a = oracle.bisect_next_beta(16, h, 0.95, 1.0, 0.1, 0.5)
    assert b == 1.0  # the whole remaining range keeps the overlap
    b, a = oracle.bisect_next_beta(16, h, 1.0, 1.0, 0.1, 0.5)
    assert b == 1.0 and a == 1.0


def test_population_proposal_uses_current_histogram():
    pa = oracle.PA(8, 2000, seed=4)
    pa.init()
    b1, a1 = pa.propose_bisect(1.0, 0.1, 0.8)
    b2, a2 = oracle.bisect_next_beta(64, pa.histogram().astype(np.int64), 0.0, 1.0, 0.1, 0.8)
    assert (b1, a1) == (b2, a2)
