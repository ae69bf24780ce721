"""Helpers that run the CUDA path and the CPU oracle on the same seeded input and compare
them: bit-exact on spin hashes, histograms, copy numbers, levels, magnetisations and family
ids; binary64 observables within 1e-12 relative (the only difference allowed is the last
ulp of ln, which comes from two different libm implementations)."""
from __future__ import annotations

import numpy as np

import oracle

FLOAT_KEYS = ("e", "C", "m", "m2", "chi", "lnQ", "minus_betaF", "rho_t", "sum_lnRratio")
REL_TOL = 1e-12


def assert_obs_close(og: dict, orf: dict, where: str = ""):
    assert og["R"] == orf["R"], where
    assert og["families"] == orf["families"], where
    assert og["step"] == orf["step"], where
    for k in FLOAT_KEYS:
        a, b = og[k], orf[k]
        assert abs(a - b) <= REL_TOL * max(1.0, abs(b)), f"{where} {k}: gpu {a!r} oracle {b!r}"
    s = orf["sums"]
    assert (og["sum_E"], og["sum_E2"], og["sum_absM"], og["sum_M2"], og["sum_size2"]) == \
        (s[0], s[1], s[2], s[3], s[5]), where


def compare_population(gpu, ref, where: str = "", hashes: bool = True):
    assert gpu.R == ref.R, where
    assert np.array_equal(gpu.histogram(), ref.histogram()), f"histogram {where}"
    lv, mg, fm = gpu.replicas()
    E, M, F = ref.state()
    N = ref.N
    assert np.array_equal(lv, (E + 2 * N) // 4), f"levels {where}"
    assert np.array_equal(mg, M), f"magnetisations {where}"
    assert np.array_equal(fm, F), f"family ids {where}"
    assert np.all(np.diff(fm) >= 0), f"tree order {where}"
    if hashes:
        assert np.array_equal(gpu.hashes(), ref.hashes()), f"spin hashes {where}"


def run_side_by_side(gpu, ref, betas, theta, check_every: int = 1):
    """Anneal both through `betas` (steps 1..n) comparing everything at every step."""
    ref.init()
    compare_population(gpu, ref, "after init")
    assert_obs_close(gpu.observables(), ref.observables(), "after init")
    for i, beta in enumerate(betas, start=1):
        gpu.resample(beta)
        st = ref.resample(beta)
        assert st == 0
        assert np.array_equal(gpu.copy_counts(), ref.counts()), f"copy numbers step {i}"
        gpu.anneal_step(theta)
        ref.sweep(theta)
        if i % check_every == 0 or i == len(betas):
            compare_population(gpu, ref, f"step {i}")
            assert_obs_close(gpu.observables(), ref.observables(), f"step {i}")


def spins_from_canonical(L: int, words: np.ndarray) -> np.ndarray:
    """(count, L, ceil(L/32)) canonical words -> (count, L*L) int8 spins."""
    out = np.empty((words.shape[0], L * L), np.int8)
    for j in range(words.shape[0]):
        out[j] = oracle.unpack(L, words[j].reshape(-1))
    return out
