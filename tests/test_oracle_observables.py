"""Pins of the oracle's population averages (Sec. III: e, C, m = <|M|>/N, <m^2> = <M^2>/N^2,
chi = beta N (<m^2> - m^2)) and family statistics (Sec. V, Eq. rhot) against values fixed by
hand and by exact enumeration, so that a slip in a formula (N instead of N^2, the signed
magnetisation in chi, a family run miscounted) fails here and not only on both sides of a
GPU comparison."""
import math

import numpy as np
import pytest

import oracle

LN2 = math.log(2.0)


def _population_L4():
    """Four hand-built 4x4 replicas with known E and M:
    all up (E=-32, M=16), all down (E=-32, M=-16), rows 0-1 up / rows 2-3 down (two straight
    domain walls of 4 bonds each: E=-32+2*8=-16, M=0), checkerboard (E=+32, M=0)."""
    L = 4
    up = np.ones((L, L), np.int8)
    stripes = np.ones((L, L), np.int8)
    stripes[2:, :] = -1
    r, c = np.indices((L, L))
    check = np.where((r + c) % 2 == 0, 1, -1).astype(np.int8)
    return L, np.stack([up, -up, stripes, check])


def test_hand_built_population_observables():
    """Sums worked out by hand for the four replicas above at beta = 0.5:
    sum E = -48, sum E^2 = 3328, sum |M| = 32, sum M^2 = 512 (R = 4, N = 16), so
    e = -0.75, C = 0.25 (832 - 144) / 16 = 10.75, m = 0.5, <m^2> = 0.5, chi = 8 (0.5 - 0.25) = 2.
    Family ids 0, 0, 1, 3: f = 3 families of sizes 2, 1, 1, rho_t = (4 + 1 + 1) / 4 = 1.5.
    -beta F = N ln 2 + sum ln Q (Sec. VII) with sum ln Q = 0.7."""
    L, spins = _population_L4()
    pa = oracle.PA(L, 4, seed=1)
    pa.set_population(spins, np.array([0, 0, 1, 3], np.int32), step=3, beta=0.5, sum_lnQ=0.7)
    E, M, _ = pa.state()
    assert E.tolist() == [-32, -32, -16, 32] and M.tolist() == [16, -16, 0, 0]
    o = pa.observables()
    assert o["R"] == 4
    assert o["e"] == -0.75
    assert o["C"] == 10.75
    assert o["m"] == 0.5           # a signed mean would give 0
    assert o["m2"] == 0.5          # dividing <M^2> by N instead of N^2 would give 8
    assert o["chi"] == 2.0         # chi from the signed mean would give 4
    assert o["families"] == 3
    assert o["rho_t"] == 1.5
    assert o["minus_betaF"] == 16 * LN2 + 0.7
    assert o["sums"].tolist() == [-48, 3328, 32, 512, 3, 6]


def test_rho_t_of_hand_built_families():
    """rho_t = R * sum_k (size_k / R)^2 (Eq. rhot) and f for family layouts worked out by hand:
    one family (rho_t = R), all singletons (rho_t = 1), sizes 3, 1, 2 (rho_t = 14/6), and a
    layout whose neighbouring runs share no id but whose ids are not consecutive."""
    L = 4
    N = L * L
    cases = [([5] * 6, 1, 6.0), (list(range(6)), 6, 1.0), ([0, 0, 0, 4, 7, 7], 3, 14.0 / 6.0),
             ([2, 9, 9, 9, 9, 11], 3, 18.0 / 6.0)]
    rng = np.random.default_rng(3)
    for fam, f_want, rho_want in cases:
        spins = np.where(rng.random((6, L, L)) < 0.5, 1, -1).astype(np.int8)
        pa = oracle.PA(L, 6, seed=1)
        pa.set_population(spins, np.array(fam, np.int32), step=1, beta=0.3)
        o = pa.observables()
        assert o["families"] == f_want, fam
        assert o["rho_t"] == pytest.approx(rho_want, rel=1e-15), fam
        assert o["R"] == 6 and N == 16


def test_bruteforce_magnetisation_sums_closed_forms():
    """The enumeration's per-level sums of |M| and M^2 (used as the exact reference below)
    against closed forms: over all 2^N states sum M^2 = 2^N N (independent +-1 spins) and
    sum |M| = sum_j C(N, j) |2j - N|; the two ground states (level 0) have |M| = N; the
    checkerboard pair (level N) has M = 0; per level |M| <= N and M^2 <= N |M|."""
    L = 4
    N = L * L
    g, sa, s2 = oracle.bruteforce(L)
    assert g.sum() == 2 ** N
    assert s2.sum() == 2 ** N * N
    assert sa.sum() == sum(math.comb(N, j) * abs(2 * j - N) for j in range(N + 1))
    assert g[0] == 2 and sa[0] == 2 * N and s2[0] == 2 * N * N
    assert g[N] == 2 and sa[N] == 0 and s2[N] == 0
    assert np.all(sa <= N * g) and np.all(s2 <= N * sa)


def _exact_L4(beta, g, sa, s2):
    N = 16
    Ek = (4 * np.arange(N + 1) - 2 * N).astype(float)
    w = g * np.exp(-beta * (Ek - Ek.min()))
    Z = w.sum()
    absM = (sa * np.exp(-beta * (Ek - Ek.min()))).sum() / Z
    M2 = (s2 * np.exp(-beta * (Ek - Ek.min()))).sum() / Z
    return absM, M2


@pytest.mark.slow
@pytest.mark.parametrize("update", [oracle.METROPOLIS, oracle.HEATBATH])
def test_anneal_L4_magnetisation_matches_enumeration(update):
    """Along a whole L=4 anneal the population's m, <m^2> and chi agree with the exact
    thermal averages from enumeration (<|M|>, <M^2> per level), within a few standard
    errors estimated from the population itself with R_eff = R / rho_t (Eq. rhot)."""
    L, R, theta = 4, 20000, 5
    N = L * L
    g, sa, s2 = oracle.bruteforce(L)
    pa = oracle.PA(L, R, seed=41, update=update)
    pa.init()
    for i in range(1, 21):
        beta = i / 20.0
        assert pa.resample(beta) == 0
        pa.sweep(theta)
        o = pa.observables()
        _, M, _ = pa.state()
        aM = np.abs(M.astype(np.float64))
        reff = o["R"] / o["rho_t"]
        absM, M2 = _exact_L4(beta, g, sa, s2)
        m_ex, m2_ex = absM / N, M2 / N ** 2
        chi_ex = beta * N * (m2_ex - m_ex ** 2)
        se_m = aM.std() / N / math.sqrt(reff)
        se_m2 = (aM ** 2).std() / N ** 2 / math.sqrt(reff)
        assert abs(o["m"] - m_ex) < 6 * se_m + 1e-12, (beta, o["m"], m_ex)
        assert abs(o["m2"] - m2_ex) < 6 * se_m2 + 1e-12, (beta, o["m2"], m2_ex)
        se_chi = beta * N * (se_m2 + 2 * m_ex * se_m)
        assert abs(o["chi"] - chi_ex) < 6 * se_chi + 1e-12, (beta, o["chi"], chi_ex)
