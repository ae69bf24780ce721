"""CUDA path vs CPU oracle, element by element, through the C ABI.

Small runs are compared in full at every step; full-size populations (R = 1e5 at L = 32,
R = 1e6 at L = 64) are compared by replay: the oracle recomputes the whole resampling from
the device's pre-resampling levels, and re-sweeps a deterministic sample of replica slots
from their exported pre-sweep spins.
"""
import math

import numpy as np
import pytest

import oracle
from side_by_side import (assert_obs_close, compare_population, run_side_by_side,
                          spins_from_canonical)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pa(*a, **k):
    from paper_2102_06611_gb300 import PopulationAnnealing
    return PopulationAnnealing(*a, **k)


# ------------------------------------------------------------------------------ init
@pytest.mark.parametrize("L,R", [(4, 300), (8, 300), (12, 200), (16, 200), (20, 150), (24, 100), (32, 100),
                                 (40, 60), (48, 50), (64, 40), (80, 20), (96, 15), (128, 9)])
def test_init_parity(L, R):
    gpu = _pa(L, R, seed=11)
    ref = oracle.PA(L, R, seed=11)
    ref.init()
    compare_population(gpu, ref, f"init L={L}")
    assert_obs_close(gpu.observables(), ref.observables(), "init")


@pytest.mark.parametrize("L", [4, 8, 12, 20, 24, 40, 64, 80, 96, 128])
def test_sweep_at_beta_zero_inverts(L):
    """At beta = 0 every proposal is accepted: one sweep maps s -> -s (Sec. IV)."""
    gpu = _pa(L, 17, seed=2)
    before = gpu.export_spins()
    gpu.anneal_step(1)
    after = gpu.export_spins()
    # word w of a row holds columns 32 w .. 32 w + 31 (bits beyond L stay clear)
    nw = before.shape[-1]
    mask = np.array([(1 << min(32, L - 32 * w)) - 1 for w in range(nw)], dtype=np.uint64).astype(np.uint32)
    assert np.array_equal(after, (~before) & mask)


# ------------------------------------------------------------------------------ full runs
RUNS = [
    # L, R, kind, n_temperatures, theta
    (4, 500, "nearest", 21, 3),
    (8, 1000, "nearest", 101, 10),   # the L=8 / R=1000 / 101-temperature / theta=10 workload
    (8, 600, "poisson", 31, 4),
    (12, 300, "nearest", 11, 3),
    (16, 400, "poisson", 11, 3),
    (24, 200, "nearest", 8, 2),
    (32, 600, "nearest", 11, 3),
    (32, 600, "poisson", 11, 3),
    (48, 100, "nearest", 5, 2),
    (64, 150, "nearest", 5, 2),
    (128, 12, "nearest", 3, 1),
    (20, 400, "nearest", 11, 3),     # the register kernels of the sizes 20, 40, 80, 96
    (40, 200, "poisson", 8, 3),
    (80, 60, "nearest", 5, 2),
    (96, 40, "nearest", 4, 2),
]


@pytest.mark.parametrize("L,R,kind,nT,theta", RUNS)
def test_run_parity(L, R, kind, nT, theta):
    seed = 1
    gpu = _pa(L, R, seed=seed, resample=kind)
    ref = oracle.PA(L, R, seed, kind=oracle.POISSON if kind == "poisson" else oracle.NEAREST,
                    capacity=gpu.capacity)
    betas = [i / (nT - 1) for i in range(1, nT)]
    run_side_by_side(gpu, ref, betas, theta)


# Low temperatures after a fast quench: most sites have three or four aligned neighbours, so
# the top 8 bits of many uniforms tie with the threshold's (2^-8 per site) and the low 24
# bits decide.  At L = 128 (256 sites per lane) a warp often holds more than 32 tie words,
# which the tie queue resolves in several passes; L = 24 and 32 use the queue on packed
# chunks, L = 16 the per-lane loop.
TIE_HEAVY = [
    (128, 400, [0.5, 0.8, 1.0], 2),
    (64, 1500, [0.45, 0.7, 0.95], 3),
    (32, 3000, [0.5, 0.9], 3),
    (24, 3000, [0.5, 0.9], 3),
    (16, 5000, [0.5, 0.9], 3),
]


@pytest.mark.parametrize("L,R,betas,theta", TIE_HEAVY)
def test_tie_heavy_parity(L, R, betas, theta):
    gpu = _pa(L, R, seed=3)
    ref = oracle.PA(L, R, 3, capacity=gpu.capacity)
    run_side_by_side(gpu, ref, betas, theta)


def test_split_sweeps_equal_one_call():
    """Sweeps are numbered within a temperature step, so 3 + 7 sweeps == 10 sweeps."""
    L, R = 16, 200
    a = _pa(L, R, seed=5)
    b = _pa(L, R, seed=5)
    for pa in (a, b):
        pa.resample(0.3)
    a.anneal_step(3)
    a.anneal_step(7)
    b.anneal_step(10)
    assert np.array_equal(a.hashes(), b.hashes())
    ref = oracle.PA(L, R, 5)
    ref.init()
    ref.resample(0.3)
    ref.sweep(3)
    ref.sweep(7)
    assert np.array_equal(a.hashes(), ref.hashes())


def test_theta_zero_and_repeated_observables():
    gpu = _pa(8, 100, seed=3)
    gpu.resample(0.2)
    gpu.anneal_step(0)
    o1 = gpu.observables()
    o2 = gpu.observables()
    assert o1 == o2
    ref = oracle.PA(8, 100, 3)
    ref.init()
    ref.resample(0.2)
    ref.sweep(0)
    assert_obs_close(o1, ref.observables())


def test_determinism_two_runs():
    """Two identical runs give identical states (no race in atomics, scan or copy)."""
    out = []
    for _ in range(2):
        gpu = _pa(32, 3000, seed=9, resample="poisson")
        for i in range(1, 6):
            gpu.resample(i * 0.08)
            gpu.anneal_step(2)
        out.append((gpu.hashes(), gpu.histogram(), gpu.observables()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]


# ------------------------------------------------------------------------------ errors
def test_capacity_overflow_is_an_error_not_a_fault():
    from paper_2102_06611_gb300 import PAError
    gpu = _pa(4, 500, seed=1, resample="poisson", capacity=500)
    with pytest.raises(PAError) as ei:
        for i in range(1, 40):
            gpu.resample(i * 0.05)
            gpu.anneal_step(1)
            gpu.sync()
    assert ei.value.status == 3  # PA_ERR_CAPACITY
    # the context stays usable for error reporting
    assert b"capacity" in gpu.lib.pa_last_error(gpu.ctx)


def test_call_order_errors():
    from paper_2102_06611_gb300 import PAError
    gpu = _pa(8, 50, seed=1)
    gpu.resample(0.5)
    with pytest.raises(PAError) as ei:
        gpu.resample(0.4)
    assert ei.value.status == 2
    with pytest.raises(PAError):
        gpu.anneal_step(-1)
    gpu.anneal_step(1)  # still usable after argument errors
    gpu.sync()


# ------------------------------------------------------------------------------ full size
def _replay_steps(L, R, kind, seed, betas, theta, n_sample, update="metropolis", gpu=None, beta_prev=0.0,
                  first_step=1):
    """Run the device at full size; replay every resampling in full and a sample of the
    sweeps in the oracle.  With `gpu` given, continue that run (at beta_prev, next step
    first_step) instead of starting from simple sampling."""
    N = L * L
    rng = np.random.default_rng(seed + first_step)
    if gpu is None:
        gpu = _pa(L, R, seed=seed, resample=kind, update=update)
        # init: sampled slots against the oracle's init
        sample = np.unique(np.concatenate([[0, R - 1], rng.integers(0, R, n_sample)]))
        for j in sample:
            w = gpu.export_spins(int(j), 1)[0]
            assert np.array_equal(w.reshape(-1), oracle.pack(L, oracle.init_replica(L, seed, int(j)))), j
    for i, beta in enumerate(betas, start=first_step):
        lv, mg, fm = gpu.replicas()
        R_prev = len(lv)
        h = np.bincount(lv, minlength=N + 1)
        assert np.array_equal(gpu.histogram(), h)
        gpu.resample(beta)
        st, counts, lnQ, S, kmin, R_new = oracle.resample_levels(
            L, R, lv, beta_prev, beta, i, seed, oracle.POISSON if kind == "poisson" else oracle.NEAREST,
            gpu.capacity)
        assert st == 0
        assert np.array_equal(gpu.copy_counts(), counts), f"copy numbers step {i}"
        assert gpu.R == R_new
        parents = np.repeat(np.arange(R_prev), counts)
        lv2, mg2, fm2 = gpu.replicas()
        assert np.array_equal(fm2, fm[parents]) and np.array_equal(lv2, lv[parents])
        assert np.array_equal(mg2, mg[parents])
        # sweeps: sampled slots, replayed from the exported pre-sweep spins
        sample = np.unique(np.concatenate([[0, R_new - 1], rng.integers(0, R_new, n_sample)]))
        pre = {int(j): gpu.export_spins(int(j), 1) for j in sample}
        gpu.anneal_step(theta)
        obs = gpu.observables()
        assert abs(obs["lnQ"] - lnQ) <= 1e-12 * max(1.0, abs(lnQ))
        for j, w in pre.items():
            s = spins_from_canonical(L, w)[0]
            s2 = oracle.sweep_replica(L, seed, i, j, beta, theta, s,
                                      update=oracle.HEATBATH if update == "heatbath" else oracle.METROPOLIS)
            post = gpu.export_spins(j, 1)[0].reshape(-1)
            assert np.array_equal(post, oracle.pack(L, s2)), f"slot {j} step {i}"
        # observables at full size from the exact integer sums
        lv3, mg3, fm3 = gpu.replicas()
        E = 4 * lv3.astype(np.int64) - 2 * N
        assert obs["sum_E"] == int(E.sum()) and obs["sum_E2"] == int((E * E).sum())
        assert obs["sum_absM"] == int(np.abs(mg3).sum()) and obs["sum_M2"] == int((mg3.astype(np.int64) ** 2).sum())
        _, sizes = np.unique(fm3, return_counts=True)
        assert obs["families"] == len(sizes) and obs["sum_size2"] == int((sizes.astype(np.int64) ** 2).sum())
        Rd, Nd = float(R_new), float(N)
        meanE = obs["sum_E"] / Rd
        meanE2 = obs["sum_E2"] / Rd
        assert obs["e"] == meanE / Nd
        assert obs["C"] == ((beta * beta) * (meanE2 - meanE * meanE)) / Nd
        beta_prev = beta
    return gpu


@pytest.mark.parametrize("kind", ["nearest", "poisson"])
def test_full_size_L32_R1e5_replay(kind):
    _replay_steps(32, 100_000, kind, seed=1, betas=[0.005, 0.01, 0.015], theta=10, n_sample=48)


def test_full_size_L64_R1e6_replay():
    _replay_steps(64, 1_000_000, "nearest", seed=7, betas=[1 / 300, 2 / 300], theta=10, n_sample=24)


def test_full_size_L64_R1e6_heatbath_replay():
    _replay_steps(64, 1_000_000, "nearest", seed=7, betas=[0.3, 0.7], theta=10, n_sample=24, update="heatbath")


@pytest.mark.parametrize("update", ["metropolis", "heatbath"])
def test_full_size_L64_R1e6_low_temperature_replay(update):
    """The headline population at the critical point and deep in the ordered phase, where most
    sites have all four neighbours aligned and the Metropolis decisions hinge on the rare
    random numbers below e^{-8 beta} (ties of the top bits are frequent): a short anneal on the
    headline schedule (theta = 1) reaches beta = 0.44 and 0.9, then two steps each are replayed
    with 512 sampled slots and the whole resampling."""
    L, R, seed, theta = 64, 1_000_000, 7, 10
    gpu = _pa(L, R, seed=seed, update=update)
    i = 0
    for target in (132, 270):                       # beta = i / 300: 0.44, 0.9
        while i < target:
            i += 1
            gpu.resample(i / 300)
            gpu.anneal_step(1)
        _replay_steps(L, R, "nearest", seed, [(i + 1) / 300, (i + 2) / 300], theta, 512, update=update, gpu=gpu,
                      beta_prev=i / 300, first_step=i + 1)
        i += 2


def test_full_size_L128_R2e5_replay():
    """The size on which the learned and the plain schedule are compared (L = 128, R = 2e5),
    64-bit half-row words, one block per SM."""
    _replay_steps(128, 200_000, "nearest", seed=1, betas=[0.44, 0.9], theta=10, n_sample=10)
