"""Pins of the oracle's population-annealing loop (Sec. II) against exact results.

Statistical checks use fixed seeds and tolerances of several standard errors; the
standard errors are taken from the family statistics (rho_t, Eq. rhot), which bound the
loss of independent replicas through resampling.
"""
import math

import numpy as np
import pytest

import oracle

LN2 = math.log(2.0)


def _levels_energy(L, E):
    return (np.asarray(E) + 2 * L * L) // 4


def test_beta0_population_closed_forms():
    """At beta = 0 (simple sampling): <E> = 0, Var(E) = 2N (the paper's sigma_0^2 = z L^d/2
    with z = 4), <M^2> = N, -beta F_0 = N ln 2 (Sec. VII)."""
    L, R = 8, 60000
    N = L * L
    pa = oracle.PA(L, R, seed=17)
    pa.init()
    o = pa.observables()
    E, M, fam = pa.state()
    assert np.array_equal(fam, np.arange(R))
    assert o["minus_betaF"] == N * LN2
    assert abs(E.mean()) < 5 * math.sqrt(2 * N / R)
    assert E.var() == pytest.approx(2 * N, rel=5 * math.sqrt(2.0 / R))
    assert (M.astype(np.float64) ** 2).mean() == pytest.approx(N, rel=5 * math.sqrt(2.0 / R))
    assert o["families"] == R and o["rho_t"] == 1.0


def test_first_lnQ_estimates_exact_partition_ratio():
    """Q_1 estimates Z(beta_1)/Z(0) (Eq. Q and the telescoping product of Sec. VII)."""
    L, R, b1 = 4, 200000, 0.2
    pa = oracle.PA(L, R, seed=5)
    pa.init()
    E, _, _ = pa.state()
    st, counts, lnQ, S, kmin, R_new = oracle.resample_levels(L, R, _levels_energy(L, E), 0.0, b1,
                                                             1, 5, oracle.NEAREST, oracle.default_capacity(R))
    assert st == 0
    exact = oracle.kaufman_lnZ(L, b1) - 16 * LN2
    w = np.exp(-b1 * E.astype(float))
    sigma = w.std() / math.sqrt(R) / w.mean()
    assert abs(lnQ - exact) < 5 * sigma
    # same quantity computed directly from the energies
    assert lnQ == pytest.approx(math.log(w.mean()), rel=1e-12, abs=1e-13)


def test_thermodynamic_integration_limit():
    """For small steps ln Q -> -dbeta <E> (Sec. VII, thermodynamic-integration limit)."""
    L, R = 8, 20000
    pa = oracle.PA(L, R, seed=8)
    pa.init()
    pa.resample(0.3)
    pa.sweep(10)
    E, _, _ = pa.state()
    for db in (1e-4, 1e-5):
        _, _, lnQ, _, _, _ = oracle.resample_levels(L, R, _levels_energy(L, E), 0.3, 0.3 + db, 2, 8,
                                                    oracle.NEAREST, oracle.default_capacity(R))
        mean = E.astype(float).mean()
        var = E.astype(float).var()
        assert lnQ == pytest.approx(-db * mean + 0.5 * db * db * var, rel=1e-5, abs=1e-14)


def test_nearest_integer_counts_bounds_and_mean():
    """Eq. (resampling-factors): r_j in {floor tau, floor tau + 1}; <r_j> = tau_hat_j."""
    L, R = 8, 50000
    pa = oracle.PA(L, R, seed=9)
    pa.init()
    E, _, _ = pa.state()
    db = 0.05
    st, counts, lnQ, S, kmin, R_new = oracle.resample_levels(L, R, _levels_energy(L, E), 0.0, db, 1, 9,
                                                             oracle.NEAREST, oracle.default_capacity(R))
    w = np.exp(-db * E.astype(float))
    tau = R * w / w.sum()
    fl = np.floor(tau)
    assert np.all((counts == fl) | (counts == fl + 1))
    assert R_new == counts.sum()
    assert fl.sum() <= R_new <= fl.sum() + R
    # mean of the fractional part decision per energy
    frac = tau - fl
    extra = counts - fl
    assert abs(extra.sum() - frac.sum()) < 5 * math.sqrt(np.sum(frac * (1 - frac)))


def test_multinomial_counts_fixed_size_mean_and_variance():
    """Multinomial resampling (Sec. II): exactly R children; r_j is Binomial(R, p_j) with
    p_j = w_j / sum w, so per energy level the total copies have mean R P_k and variance
    R P_k (1 - P_k), P_k = h_k w_k / S (checked over the levels with P_k > 1e-3)."""
    L, R = 8, 50000
    pa = oracle.PA(L, R, seed=9)
    pa.init()
    E, _, _ = pa.state()
    lv = _levels_energy(L, E)
    db = 0.05
    w = np.exp(-db * E.astype(float))
    p = w / w.sum()
    sums = []
    for step in range(1, 41):
        st, counts, lnQ, S, kmin, R_new = oracle.resample_levels(L, R, lv, 0.0, db, step, 9,
                                                                 oracle.MULTINOMIAL, oracle.default_capacity(R))
        assert st == 0 and R_new == R and counts.sum() == R
        sums.append(np.bincount(lv, weights=counts, minlength=L * L + 1))
    sums = np.array(sums)
    P = np.bincount(lv, weights=p, minlength=L * L + 1)
    sel = P > 1e-3
    mean = sums[:, sel].mean(axis=0)
    var = sums[:, sel].var(axis=0, ddof=1)
    expect_var = R * P[sel] * (1 - P[sel])
    z = (mean - R * P[sel]) / np.sqrt(expect_var / len(sums))
    assert np.all(np.abs(z) < 5)
    # variance ratio: chi-square with 39 dof per level, averaged over the levels
    assert abs(np.mean(var / expect_var) - 1) < 0.25


def test_multinomial_uniform_weights_are_binomial_counts():
    """With dbeta = 0 every parent has probability 1/R: r_j ~ Binomial(R, 1/R), whose
    frequencies of 0, 1, 2, 3 copies are checked by chi-square."""
    L, R = 4, 20000
    pa = oracle.PA(L, R, seed=2)
    pa.init()
    E, _, _ = pa.state()
    st, counts, *_ = oracle.resample_levels(L, R, _levels_energy(L, E), 0.3, 0.3, 1, 2, oracle.MULTINOMIAL,
                                            oracle.default_capacity(R))
    assert counts.sum() == R
    obs = np.bincount(counts, minlength=5)[:4]
    pk = np.array([math.comb(R, k) * (1 / R) ** k * (1 - 1 / R) ** (R - k) for k in range(4)])
    chi2 = np.sum((obs - R * pk) ** 2 / (R * pk))
    assert chi2 < 3 + 6 * math.sqrt(6)


@pytest.mark.parametrize("lam", [0.3, 1.0, 2.5, 70.0])
def test_poisson_sampler_pmf(lam):
    n = 30000
    draws = np.array([oracle.poisson(lam, 77, j, 3) for j in range(n)])
    assert draws.mean() == pytest.approx(lam, abs=5 * math.sqrt(lam / n))
    assert draws.var() == pytest.approx(lam, rel=6 * math.sqrt(2.0 / n) + 5 * math.sqrt(1 / (lam * n)))
    ks = np.arange(0, int(lam + 10 * math.sqrt(lam) + 10))
    logp = -lam + ks * math.log(lam) - np.array([math.lgamma(k + 1) for k in ks])
    p = np.exp(logp)
    obs = np.bincount(draws, minlength=len(ks))[: len(ks)]
    mask = p * n > 5
    chi2 = np.sum((obs[mask] - n * p[mask]) ** 2 / (n * p[mask]))
    dof = mask.sum() - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof)


def test_poisson_counts_in_resampling_mean():
    L, R = 8, 40000
    pa = oracle.PA(L, R, seed=10, kind=oracle.POISSON)
    pa.init()
    E, _, _ = pa.state()
    db = 0.03
    st, counts, *_ = oracle.resample_levels(L, R, _levels_energy(L, E), 0.0, db, 1, 10,
                                            oracle.POISSON, 10 * R)
    w = np.exp(-db * E.astype(float))
    tau = R * w / w.sum()
    assert st == 0
    assert abs(counts.sum() - R) < 5 * math.sqrt(R)
    assert abs((counts - tau).sum()) < 5 * math.sqrt(tau.sum())


def test_tree_order_and_copies():
    """Children of one parent sit next to each other in parent order (Sec. V): family
    ids stay sorted, each child is a bit copy of its parent."""
    L, R = 8, 3000
    pa = oracle.PA(L, R, seed=12)
    pa.init()
    for i, beta in enumerate([0.1, 0.2, 0.3, 0.4], start=1):
        spins_before = pa.spins()
        _, _, fam_before = pa.state()
        assert pa.resample(beta) == 0
        counts = pa.counts()
        E, M, fam = pa.state()
        assert np.all(np.diff(fam) >= 0)
        parents = np.repeat(np.arange(len(counts)), counts)
        assert np.array_equal(pa.spins(), spins_before[parents])
        assert np.array_equal(fam, fam_before[parents])
        h = pa.histogram()
        assert h.sum() == pa.R
        pa.sweep(3)


def test_capacity_overflow_is_reported():
    L, R = 4, 500
    pa = oracle.PA(L, R, seed=1, kind=oracle.POISSON, capacity=R)
    pa.init()
    sts = [pa.resample(b) for b in (0.5, 1.0, 1.5, 2.0)]
    assert 3 in sts  # Poisson population exceeds a capacity of exactly R at some step


@pytest.mark.slow
@pytest.mark.parametrize("update,kind", [(oracle.METROPOLIS, oracle.NEAREST), (oracle.HEATBATH, oracle.NEAREST),
                                         (oracle.METROPOLIS, oracle.MULTINOMIAL)])
def test_full_anneal_L4_matches_enumeration(update, kind):
    """A whole anneal at L=4 reproduces the exact ln Z (Sec. VII estimator), <E> and C
    within a few standard errors, with the Metropolis and the heatbath update (Sec. IV) and
    with nearest-integer and multinomial resampling (Sec. II)."""
    L, R, theta = 4, 20000, 5
    N = L * L
    g, _, _ = oracle.bruteforce(L)
    Ek = (4 * np.arange(N + 1) - 2 * N).astype(float)
    pa = oracle.PA(L, R, seed=31, kind=kind, update=update)
    pa.init()
    for i in range(1, 21):
        beta = i / 20.0
        assert pa.resample(beta) == 0
        pa.sweep(theta)
        o = pa.observables()
        w = g * np.exp(-beta * (Ek - Ek.min()))
        Z = w.sum()
        mE = (w * Ek).sum() / Z
        varE = (w * Ek * Ek).sum() / Z - mE ** 2
        lnZ = math.log(Z) - beta * Ek.min()
        reff = o["R"] / o["rho_t"]
        se_e = math.sqrt(varE / reff) / N
        assert abs(o["e"] - mE / N) < 6 * se_e + 1e-12, (beta, o["e"], mE / N)
        assert abs(o["minus_betaF"] - lnZ) < 0.02, (beta, o["minus_betaF"], lnZ)
        C = beta ** 2 * varE / N
        assert abs(o["C"] - C) < 0.1 * C + 0.02


@pytest.mark.slow
@pytest.mark.parametrize("update", [oracle.METROPOLIS, oracle.HEATBATH])
def test_anneal_L8_against_kaufman(update):
    L, R, theta = 8, 5000, 10
    N = L * L
    pa = oracle.PA(L, R, seed=1, update=update)
    pa.init()
    for i in range(1, 51):
        beta = i / 50.0
        assert pa.resample(beta) == 0
        pa.sweep(theta)
    o = pa.observables()
    e_ex, c_ex, lnZ = oracle.kaufman_thermo(L, 1.0)
    assert abs(o["e"] - e_ex / N) < 0.01
    assert abs(o["minus_betaF"] - lnZ) / N < 2e-3


@pytest.mark.slow
@pytest.mark.parametrize("L,update", [(6, oracle.HEATBATH), (10, oracle.METROPOLIS)])
def test_anneal_padded_rows_against_exact(L, update):
    """Sizes whose half-rows are padded in the random-number chunks (L/2 = 3, 5 sites in
    H' = 4, 8 bit positions, several rows per chunk, the last chunk partial): whole anneals
    reproduce Kaufman's exact free energy along the way and the energy at beta = 1."""
    R, theta, n = 800, 5, 20
    N = L * L
    pa = oracle.PA(L, R, seed=5, update=update)
    pa.init()
    for i in range(1, n + 1):
        beta = i / n
        assert pa.resample(beta) == 0
        pa.sweep(theta)
        if i in (8, 12, 16):
            o = pa.observables()
            assert abs(o["minus_betaF"] - oracle.kaufman_lnZ(L, beta)) / N < 5e-3, (L, beta)
    o = pa.observables()
    e_ex, _, lnZ = oracle.kaufman_thermo(L, 1.0)
    assert abs(o["e"] - e_ex / N) < 0.01
    assert abs(o["minus_betaF"] - lnZ) / N < 5e-3


@pytest.mark.parametrize("kind", [oracle.NEAREST, oracle.POISSON, oracle.MULTINOMIAL])
def test_resample_shard_equals_whole_population(kind):
    """Copy numbers drawn shard by shard (tables from the whole histogram, parents keyed by
    their global index; multinomial: the children whose draw falls in the shard's range of the
    running weight sum) are those of the whole population (Sec. II), for any split; ln Q_i
    is the whole population's."""
    L, R = 8, 4000
    pa = oracle.PA(L, R, seed=21)
    pa.init()
    E, _, _ = pa.state()
    levels = _levels_energy(L, E).astype(np.int32)
    hist = np.bincount(levels, minlength=L * L + 1)
    st, counts, lnQ, _, _, R_new = oracle.resample_levels(L, R, levels, 0.0, 0.35, 1, 21, kind,
                                                          oracle.default_capacity(R))
    assert st == 0
    for cuts in ([0, R], [0, 1234, R], [0, 1, 2, 2999, R], [0, 1000, 1000, 2500, R]):
        parts, total = [], 0
        for a, b in zip(cuts[:-1], cuts[1:]):
            before = np.bincount(levels[:a], minlength=L * L + 1)
            s, c, q, n = oracle.resample_shard(L, R, hist, R, levels[a:b], a, 0.0, 0.35, 1, 21, kind,
                                               hist_before=before)
            assert s == 0 and q == lnQ
            parts.append(c)
            total += n
        assert np.array_equal(np.concatenate(parts), counts) and total == R_new
