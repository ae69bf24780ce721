"""Pins of the CPU oracle's primitives against definitions outside the oracle.

Each test checks the oracle against something it cannot share a mistake with: published
known-answer vectors, libm and a 60-digit decimal reference, hand-derived lattice
energies, and three mutually independent exact methods for Z.
"""
import math
import os
from decimal import Decimal, getcontext

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _ulp_diff(a: float, b: float) -> int:
    ia = np.array([a], dtype=np.float64).view(np.int64)[0]
    ib = np.array([b], dtype=np.float64).view(np.int64)[0]
    return abs(int(ia) - int(ib))


# ---------------------------------------------------------------------------- Philox
def test_philox_known_answer_vectors():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(t, 16) for t in line.split()])
    assert len(rows) == 3
    for r in rows:
        out = oracle.philox4x32_10(r[0:4], r[4:6])
        assert [int(v) for v in out] == r[6:10]


def test_philox_counter_sensitivity():
    base = oracle.philox4x32_10([1, 2, 3, 4], [5, 6])
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        assert not np.array_equal(oracle.philox4x32_10(c, [5, 6]), base)


# ---------------------------------------------------------------------------- exp
def test_exp_special_values():
    assert oracle.exp(0.0) == 1.0
    assert oracle.exp(-800.0) == 0.0
    assert math.isinf(oracle.exp(800.0))
    assert oracle.exp(1.0) == pytest.approx(math.e, rel=0, abs=4.5e-16)


def test_exp_within_one_ulp_of_libm():
    rng = np.random.default_rng(11)
    xs = np.concatenate([rng.uniform(-745.0, 709.0, 20000), rng.uniform(-50.0, 0.0, 20000),
                         rng.uniform(-1e-3, 1e-3, 5000), -4.0 * np.arange(0, 1.0, 1e-3),
                         -8.0 * np.arange(0, 1.0, 1e-3)])
    worst = 0
    for x in xs:
        a = oracle.exp(float(x))
        b = math.exp(float(x))
        if b == 0.0 or a == 0.0:
            continue
        worst = max(worst, _ulp_diff(a, b))
    assert worst <= 1


def test_exp_against_decimal_reference():
    getcontext().prec = 60
    rng = np.random.default_rng(12)
    for x in rng.uniform(-40.0, 0.5, 600):
        exact = Decimal(float(x)).exp()
        got = Decimal(oracle.exp(float(x)))
        ulp = Decimal(math.ulp(float(exact)))
        assert abs(got - exact) <= ulp  # at most 1 ulp from the true value


def test_metropolis_threshold_definition():
    assert oracle.metropolis_threshold(0.0) == 2 ** 32
    getcontext().prec = 60
    for y in [0.04, 0.4, 1.7627471740390860, 4.0, 8.0, 20.0]:
        t = oracle.metropolis_threshold(y)
        exact = (Decimal(-y).exp() * Decimal(2) ** 32)
        # floor of a value within 1 ulp of exp(-y) 2^32
        assert abs(Decimal(t) - exact) <= 1
    assert oracle.metropolis_threshold(40.0) == 0


# ---------------------------------------------------------------------------- lattice
@pytest.mark.parametrize("L", [4, 8, 12, 32])
def test_energy_closed_forms(L):
    N = L * L
    up = np.ones((L, L), np.int8)
    assert oracle.energy_mag(L, up) == (-2 * N, N)
    assert oracle.energy_mag(L, -up) == (-2 * N, -N)
    r, c = np.indices((L, L))
    af = np.where((r + c) % 2 == 0, 1, -1).astype(np.int8)
    assert oracle.energy_mag(L, af) == (2 * N, 0)
    one = up.copy()
    one[L // 2, 1] = -1
    assert oracle.energy_mag(L, one) == (-2 * N + 8, N - 2)
    stripes = np.where(c < L // 2, 1, -1).astype(np.int8)  # two straight domain walls
    assert oracle.energy_mag(L, stripes) == (-2 * N + 4 * L, 0)


def test_energy_level_parity_random():
    rng = np.random.default_rng(3)
    for L in (4, 6, 8, 10):
        N = L * L
        for _ in range(50):
            s = rng.choice(np.array([-1, 1], np.int8), size=(L, L))
            E, M = oracle.energy_mag(L, s)
            assert (E + 2 * N) % 4 == 0  # antiparallel bonds come in pairs on the torus
            assert M == int(s.sum())


def test_pack_roundtrip_and_hash():
    rng = np.random.default_rng(4)
    for L in (4, 8, 12, 40, 64, 128):
        s = rng.choice(np.array([-1, 1], np.int8), size=L * L)
        w = oracle.pack(L, s)
        assert np.array_equal(oracle.unpack(L, w), s)
        # FNV-1a 64 (Fowler, Noll, Vo) over the little-endian bytes of the packed words
        h = 0xcbf29ce484222325
        for byte in w.astype("<u4").tobytes():
            h ^= byte
            h = (h * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
        assert oracle.replica_hash(L, s) == h
    # FNV-1a 64 of the empty string is the offset basis; of "a" it is the published value
    h = 0xcbf29ce484222325 ^ ord("a")
    assert (h * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF == 0xaf63dc4c8601ec8c


def test_init_bit_map_follows_stream_definition():
    L, seed = 12, 99
    for j in (0, 1, 7):
        s = oracle.init_replica(L, seed, j)
        for n in range(L * L):
            w = n >> 5
            x = oracle.philox4x32_10([w >> 2, j, 0, 0], [seed & 0xFFFFFFFF, seed >> 32])[w & 3]
            assert s[n] == (1 if (int(x) >> (n & 31)) & 1 else -1)


def test_init_is_uniform():
    L, seed = 8, 5
    tot = np.array([oracle.init_replica(L, seed, j) for j in range(2000)])
    frac = (tot > 0).mean()
    assert abs(frac - 0.5) < 5 * math.sqrt(0.25 / tot.size)


# ---------------------------------------------------------------------------- sweep
@pytest.mark.parametrize("L,r,p", [(4, 3, 1), (8, 3, 2), (12, 5, 4), (24, 23, 11), (32, 7, 9), (48, 47, 23),
                                   (64, 63, 31), (128, 5, 40), (128, 127, 63)])
def test_sweep_uniform_follows_its_definition(L, r, p):
    """Top 8 bits from bit n mod 32 of eight Philox words (bit planes) of chunk n / 32, with
    n = r H' + p the site's colour index (rows padded to H', the power of two >= L/2), low 24
    bits from a separate refinement draw, as documented in the oracle."""
    seed, step, slot, tag = 0x1234_5678_9ABC, 17, 4242, 7
    key = [seed & 0xFFFFFFFF, seed >> 32]
    hp = 1 << max(0, (L // 2 - 1).bit_length())
    n = r * hp + p
    chunk, b = n // 32, n % 32
    planes = np.concatenate([oracle.philox4x32_10([2 * chunk + c, slot, (1 << 28) | tag, step], key)
                             for c in (0, 1)])
    top = 0
    for k in range(8):
        top |= ((int(planes[k]) >> b) & 1) << (31 - k)
    low = int(oracle.philox4x32_10([64 * r + p, slot, (4 << 28) | tag, step], key)[0]) & 0xFFFFFF
    assert oracle.sweep_uniform(L, seed, step, slot, tag, r, p) == top | low


@pytest.mark.parametrize("L", [4, 8, 12, 16, 24, 32, 48, 64, 128])
def test_sweep_planes_are_distinct_per_site(L):
    """No two sites of one colour share a plane bit: two sites that did would have equal top
    bytes in every sweep, while independent ones agree in a given sweep with probability
    1/256 only."""
    seed, step, slot = 99, 3, 11
    H = L // 2
    tops = np.array([[oracle.sweep_uniform(L, seed, step, slot, tag, r, p) >> 24
                      for r in range(min(L, 8)) for p in range(H)] for tag in range(40)], dtype=np.int64)
    # sites that shared a plane bit would have identical top bytes in every draw
    n = tops.shape[1]
    same = (tops[:, :, None] == tops[:, None, :]).all(axis=0)
    assert not same[~np.eye(n, dtype=bool)].any()


def test_sweep_uniform_is_uniform():
    xs = np.array([oracle.sweep_uniform(64, 3, 1, j, t, r, p) for j in range(4) for t in range(2)
                   for r in range(64) for p in range(32)], dtype=np.uint64)
    n = len(xs)
    assert abs(xs.astype(float).mean() / 2 ** 32 - 0.5) < 5 * math.sqrt(1 / 12 / n)
    for shift, bins in ((24, 256), (0, 256)):
        counts = np.bincount(((xs >> shift) & 255).astype(np.int64), minlength=bins)
        chi2 = np.sum((counts - n / bins) ** 2 / (n / bins))
        assert chi2 < bins - 1 + 6 * math.sqrt(2 * (bins - 1))


@pytest.mark.parametrize("L", [4, 8, 12])
def test_sweep_beta_zero_inverts_every_spin(L):
    """At beta = 0 every proposal is accepted, so one checkerboard sweep maps s -> -s
    (the non-ergodicity the paper discusses for sequential updates, Sec. IV)."""
    s = oracle.init_replica(L, 3, 0)
    one = oracle.sweep_replica(L, 3, 1, 0, 0.0, 1, s)
    assert np.array_equal(one, -s)
    two = oracle.sweep_replica(L, 3, 1, 0, 0.0, 2, s)
    assert np.array_equal(two, s)


def test_sweep_frozen_ground_state():
    L = 8
    s = np.ones(L * L, np.int8)
    out = oracle.sweep_replica(L, 1, 1, 0, 10.0, 5, s)  # threshold floor(e^-80 2^32) = 0
    assert np.array_equal(out, s)


def test_sweep_single_defect_always_heals_at_zero_cost():
    """A site with a <= 2 aligned neighbours flips with probability one."""
    L = 8
    s = np.ones((L, L), np.int8)
    s[2, 2] = -1  # colour 0 site with 0 aligned neighbours
    out = oracle.sweep_replica(L, 1, 1, 0, 100.0, 1, s.ravel())
    assert np.array_equal(out, np.ones(L * L, np.int8))


def _exact_level_distribution(beta):
    g, _, _ = oracle.bruteforce(4)
    E = 4 * np.arange(17) - 32
    w = g * np.exp(-beta * (E - E.min()))
    return w / w.sum()


@pytest.mark.parametrize("beta", [0.3, 0.44, 0.7])
def test_sweep_samples_boltzmann_distribution_L4(beta):
    """Long checkerboard Metropolis chains at L=4 reproduce the exact level distribution
    from enumeration (chi-square with the correlated-sample allowance of a 6 sigma cut)."""
    L, seed, reps, blocks, theta = 4, 21, 400, 30, 6
    counts = np.zeros(17)
    for j in range(reps):
        s = oracle.init_replica(L, seed, j)
        for blk in range(1, blocks + 1):
            s = oracle.sweep_replica(L, seed, blk, j, beta, theta, s)
            E, _ = oracle.energy_mag(L, s)
            counts[(E + 32) // 4] += 1
    p = _exact_level_distribution(beta)
    n = counts.sum()
    mask = p * n > 5
    chi2 = np.sum((counts[mask] - n * p[mask]) ** 2 / (n * p[mask]))
    dof = mask.sum() - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof), (chi2, dof)


# ---------------------------------------------------------------------------- exact Z
def test_enumeration_low_energy_counts():
    """Hand-derived counts at L = 4: two ground states; no state with two antiparallel
    bonds; 2 x 16 single flips (four broken bonds); 2 x 32 flipped nearest-neighbour pairs
    (six broken bonds); total 2^16; g symmetric under E -> -E (bipartite lattice)."""
    g, sa, s2 = oracle.bruteforce(4)
    assert g.sum() == 2 ** 16
    assert list(g[:4]) == [2, 0, 32, 64]
    assert np.array_equal(g, g[::-1])
    assert sa[0] == 2 * 16 and s2[0] == 2 * 256


@pytest.mark.parametrize("beta", [0.05, 0.2, 0.4406867935097715, 0.55, 1.0, 2.0])
def test_three_exact_methods_agree(beta):
    g, _, _ = oracle.bruteforce(4)
    E = 4 * np.arange(17) - 32
    lnZ_enum = math.log(float(np.sum(g * np.exp(-beta * (E - E.min()))))) - beta * E.min()
    assert oracle.transfer_lnZ(4, beta) == pytest.approx(lnZ_enum, rel=1e-13)
    assert oracle.kaufman_lnZ(4, beta) == pytest.approx(lnZ_enum, rel=1e-13)
    for L in (6, 8):
        assert oracle.kaufman_lnZ(L, beta) == pytest.approx(oracle.transfer_lnZ(L, beta), rel=1e-12)


@pytest.mark.parametrize("L", [4, 16, 64, 128])
def test_kaufman_limits(L):
    N = L * L
    assert oracle.kaufman_lnZ(L, 1e-7) == pytest.approx(N * math.log(2.0), rel=1e-9)
    b = 4.0
    assert oracle.kaufman_lnZ(L, b) == pytest.approx(2 * N * b + math.log(2.0), rel=1e-12)


def test_kaufman_thermo_matches_enumeration():
    g, _, _ = oracle.bruteforce(4)
    E = (4 * np.arange(17) - 32).astype(float)
    for beta in (0.2, 0.44, 0.8):
        w = g * np.exp(-beta * (E - E.min()))
        Z = w.sum()
        mE = (w * E).sum() / Z
        mE2 = (w * E * E).sum() / Z
        C = beta ** 2 * (mE2 - mE ** 2) / 16
        e, c, _ = oracle.kaufman_thermo(4, beta)
        assert e == pytest.approx(mE, rel=1e-9, abs=1e-9)
        assert c == pytest.approx(C, rel=1e-7)


def test_specific_heat_peak_near_onsager_point():
    """The finite-lattice C(beta) at L=64 peaks within a few 1/L of
    beta_c = ln(1 + sqrt 2) / 2 (Sec. III)."""
    bc = 0.5 * math.log(1 + math.sqrt(2))
    bs = np.linspace(0.40, 0.48, 161)
    cs = [oracle.kaufman_thermo(64, b)[1] for b in bs]
    peak = bs[int(np.argmax(cs))]
    assert abs(peak - bc) < 0.01


# ---------------------------------------------------------------------------- heatbath
def test_heatbath_thresholds():
    """T_3, T_4 = floor(2^32 / (1 + e^{4 beta})), floor(2^32 / (1 + e^{8 beta})) within the 1-ulp
    exp; beta = 0 gives 2^31 (p = 1/2); the pairs T_a + T_{4-a} = 2^32 make the flip
    probabilities of a and 4 - a complementary, and T_a / T_{4-a} = e^{-beta dE_a} is
    detailed balance of the heatbath rule (Sec. IV)."""
    getcontext().prec = 60
    assert oracle.heatbath_threshold(0.0) == 2 ** 31
    for beta in [0.05, 0.2, 0.4406867935097715, 0.9, 2.0]:
        T3, T4 = oracle.heatbath_threshold(4 * beta), oracle.heatbath_threshold(8 * beta)
        for T, y in ((T3, 4 * beta), (T4, 8 * beta)):
            exact = Decimal(2) ** 32 / (1 + Decimal(y).exp())
            assert abs(Decimal(T) - exact) <= 1
        T1, T0 = 2 ** 32 - T3, 2 ** 32 - T4
        # exact up to the floor of T_3, T_4 (one unit in the numerator)
        assert abs(T3 / T1 - math.exp(-4 * beta)) <= 2 / T1
        assert abs(T4 / T0 - math.exp(-8 * beta)) <= 2 / T0


@pytest.mark.parametrize("beta", [0.25, 0.4406867935097715, 0.7])
def test_heatbath_sweep_samples_boltzmann_distribution_L4(beta):
    """Long checkerboard heatbath chains at L=4 reproduce the exact level distribution from
    enumeration (chi-square with a 6 sigma cut)."""
    L, seed, reps, blocks, theta = 4, 23, 400, 30, 6
    counts = np.zeros(17)
    for j in range(reps):
        s = oracle.init_replica(L, seed, j)
        for blk in range(1, blocks + 1):
            s = oracle.sweep_replica(L, seed, blk, j, beta, theta, s, update=oracle.HEATBATH)
            E, _ = oracle.energy_mag(L, s)
            counts[(E + 32) // 4] += 1
    p = _exact_level_distribution(beta)
    n = counts.sum()
    mask = p * n > 5
    chi2 = np.sum((counts[mask] - n * p[mask]) ** 2 / (n * p[mask]))
    dof = mask.sum() - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof), (chi2, dof)


def test_heatbath_at_beta_zero_is_a_fair_coin_per_site():
    """At beta = 0 every site flips with probability 1/2 (x < 2^31: the top bit of its
    uniform), so one sweep flips about half the spins, unlike Metropolis which flips all."""
    L = 16
    s = oracle.init_replica(L, 3, 0)
    flips = 0
    for step in range(1, 41):
        t = oracle.sweep_replica(L, 3, step, 0, 0.0, 1, s, update=oracle.HEATBATH)
        flips += int((t != s).sum())
    n = 40 * L * L
    assert abs(flips / n - 0.5) < 5 * math.sqrt(0.25 / n)
