"""Pins of the oracle's population analysis (Sec. IV: blocked and jackknife errors, R_eff;
Sec. V: family entropy S_f and rho_s) against hand-computed cases, exact identities and
closed forms."""
import math

import numpy as np
import pytest

import oracle


def test_hand_computed_four_replicas():
    """E = (0, 4, 8, 12) in two blocks {0, 4}, {8, 12}: block means 2 and 10, so
    sigma^2_B = ((2-6)^2 + (10-6)^2) / (2 * 1) = 16; leave-one-block-out means 10 and 2, so
    sigma^2_J = (1/2) ((10-6)^2 + (2-6)^2) = 16; sigma^2(E) = (36+4+4+36)/3 = 80/3, so
    R_eff = 5/3.  C = beta^2 (<E^2> - <E>^2) / N = 0.25 (56 - 36) / 16 = 0.3125, and both
    leave-one-block-out halves give C = 0.0625, so its jackknife variance is 0.  Two
    families of two: S_f = ln 2, rho_s = 2."""
    r = oracle.analysis(16, 0.5, [0, 4, 8, 12], [4, -4, 2, 0], [0, 0, 1, 1], 2)
    assert r["mean_E"] == 6.0
    assert r["var_E"] == pytest.approx(80 / 3, rel=1e-15)
    assert r["var_mean_E_blocked"] == 16.0 and r["var_mean_E_jack"] == 16.0
    assert r["R_eff_E"] == pytest.approx(5 / 3, rel=1e-15)
    assert r["C"] == 0.3125 and r["var_C_jack"] == 0.0
    assert r["S_f"] == pytest.approx(math.log(2), rel=1e-15) and r["rho_s"] == pytest.approx(2.0, rel=1e-15)
    # |M| = (4, 4, 2, 0): blocks 4 and 1, mean 2.5
    assert r["mean_absM"] == 2.5 and r["var_mean_absM_blocked"] == pytest.approx(((4 - 2.5) ** 2 + (1 - 2.5) ** 2) / 2)
    assert r["families"] == 2


def test_jackknife_equals_blocked_for_the_mean_with_equal_blocks():
    """For a mean, leave-one-block-out values are O^J_b = (n mean - O^B_b) / (n - 1), so the
    jackknife variance equals the blocked one exactly when all blocks have equal size."""
    rng = np.random.default_rng(5)
    R, n = 6000, 100
    E = rng.integers(-500, 500, R).astype(np.int32)
    M = rng.integers(-300, 300, R).astype(np.int32)
    r = oracle.analysis(64, 0.4, E, M, np.arange(R, dtype=np.int32), n)
    assert r["var_mean_E_jack"] == pytest.approx(r["var_mean_E_blocked"], rel=1e-11)
    assert r["var_mean_absM_jack"] == pytest.approx(r["var_mean_absM_blocked"], rel=1e-11)


@pytest.mark.parametrize("R,n", [(1000, 10), (5000, 100)])
def test_block_constant_series_closed_form(R, n):
    """O constant within each of n equal blocks (perfectly correlated families): then
    sigma^2(mean) = (1/(n(n-1))) sum (v_b - v)^2 and sigma^2(O) = B sum (v_b - v)^2 / (R - 1),
    so R_eff = R (n - 1) / (R - 1) whatever the block values."""
    rng = np.random.default_rng(1)
    vals = rng.integers(-1000, 1000, n)
    E = np.repeat(vals, R // n).astype(np.int32)
    M = np.repeat(rng.integers(0, 500, n), R // n).astype(np.int32)
    r = oracle.analysis(64, 0.3, E, M, np.repeat(np.arange(n), R // n).astype(np.int32), n)
    assert r["R_eff_E"] == pytest.approx(R * (n - 1) / (R - 1), rel=1e-10)
    assert r["R_eff_M"] == pytest.approx(R * (n - 1) / (R - 1), rel=1e-10)
    assert r["families"] == n and r["S_f"] == pytest.approx(math.log(n), rel=1e-12)


def test_independent_replicas_have_R_eff_close_to_R():
    """Independent draws: E[sigma^2_J(mean)] = sigma^2 / R, so R_eff / R = 1 within the
    relative error of a variance estimated from n - 1 = 99 degrees of freedom."""
    rng = np.random.default_rng(3)
    R, n = 20000, 100
    for trial in range(3):
        E = rng.normal(0, 300, R).round().astype(np.int32)
        M = rng.integers(-1000, 1000, R).astype(np.int32)
        r = oracle.analysis(1024, 0.2, E, M, np.arange(R, dtype=np.int32), n)
        tol = 5 * math.sqrt(2 / (n - 1))
        assert abs(r["R_eff_E"] / R - 1) < tol and abs(r["R_eff_M"] / R - 1) < tol


def test_jackknife_variance_of_C_for_gaussian_energies():
    """For normal E the sample variance has variance 2 sigma^4 / (R - 1), so
    sigma^2(C) ~ beta^4 2 sigma^4 / (R N^2) for C = beta^2 Var(E) / N."""
    rng = np.random.default_rng(11)
    R, n, N, beta, sig = 40000, 100, 256, 0.4, 200.0
    E = rng.normal(0, sig, R).round().astype(np.int32)
    r = oracle.analysis(N, beta, E, np.zeros(R, np.int32), np.arange(R, dtype=np.int32), n)
    expect = beta ** 4 * 2 * sig ** 4 / (R * N * N)
    assert r["var_C_jack"] == pytest.approx(expect, rel=0.6)
    assert r["C"] == pytest.approx(beta * beta * sig * sig / N, rel=0.05)


def test_family_entropy_limits():
    """All singletons: S_f = ln R, rho_s = 1; one family: S_f = 0, rho_s = R; k equal
    families: S_f = ln k, rho_s = R / k (Sec. V, Eq. rhos)."""
    R = 1200
    E = np.zeros(R, np.int32)
    r = oracle.analysis(16, 0.1, E, E, np.arange(R, dtype=np.int32), 10)
    assert r["S_f"] == pytest.approx(math.log(R), rel=1e-12) and r["rho_s"] == pytest.approx(1.0, rel=1e-12)
    r = oracle.analysis(16, 0.1, E, E, np.zeros(R, np.int32), 10)
    assert r["S_f"] == 0.0 and r["rho_s"] == R and r["families"] == 1
    r = oracle.analysis(16, 0.1, E, E, np.repeat(np.arange(8), R // 8).astype(np.int32), 10)
    assert r["S_f"] == pytest.approx(math.log(8), rel=1e-12) and r["rho_s"] == pytest.approx(R / 8, rel=1e-12)


def test_uneven_blocks_and_arguments():
    """R not divisible by n: blocks of floor/ceil(R/n) replicas cover every replica once
    (the jackknife mean of the leave-one-out means of a constant series is that constant);
    n outside [2, R] is rejected."""
    R = 1003
    E = np.full(R, -40, np.int32)
    r = oracle.analysis(16, 0.2, E, E, np.arange(R, dtype=np.int32), 10)
    assert r["mean_E"] == -40.0 and r["var_mean_E_jack"] == 0.0 and r["var_mean_E_blocked"] == 0.0
    with pytest.raises(ValueError):
        oracle.analysis(16, 0.2, E, E, np.arange(R, dtype=np.int32), 1)
    with pytest.raises(ValueError):
        oracle.analysis(16, 0.2, E[:5], E[:5], np.arange(5, dtype=np.int32), 6)


def test_population_at_beta_zero_is_uncorrelated():
    """Right after simple sampling every replica is independent, so R_eff(E) is close to R,
    and every replica is its own family."""
    pa = oracle.PA(8, 4000, 9)
    pa.init()
    r = pa.analysis(100)
    assert abs(r["R_eff_E"] / 4000 - 1) < 5 * math.sqrt(2 / 99)
    assert r["families"] == 4000 and r["rho_s"] == pytest.approx(1.0, rel=1e-12)
