"""Population analysis on the GPU (pa_analyze) against the oracle: blocked and jackknife
errors, R_eff(E), R_eff(|M|), the jackknife error of C and the family entropy (Sec. IV,
Sec. V), at every checked step of side-by-side runs and on a full-size population."""
import math

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = ["mean_E", "var_E", "var_mean_E_jack", "var_mean_E_blocked", "R_eff_E", "mean_absM", "var_absM",
          "var_mean_absM_jack", "var_mean_absM_blocked", "R_eff_M", "C", "var_C_jack", "S_f", "rho_s"]


def _pa(*a, **k):
    from paper_2102_06611_gb300 import PopulationAnnealing
    return PopulationAnnealing(*a, **k)


def assert_analysis_close(g: dict, o: dict, where: str):
    """Block sums are exact integers and the binary64 formulas run in the same order on both
    sides; only the family-entropy sum (by family size on the GPU, family by family in the
    oracle) and libm's vs CUDA's log differ in rounding: 1e-12 relative."""
    assert g["families"] == int(o["families"]), where
    assert g["n_blocks"] == int(o["n_blocks"]), where
    for k in FIELDS:
        a, b = g[k], o[k]
        if math.isnan(b):
            assert math.isnan(a), f"{where}: {k}"
            continue
        assert abs(a - b) <= 1e-12 * max(1.0, abs(b)), f"{where}: {k} gpu {a!r} oracle {b!r}"


@pytest.mark.parametrize("L,R,kind,nT,theta,n_blocks,every", [
    (8, 1000, "nearest", 101, 10, 100, 10),   # the L=8 / R=1000 / 101-temperature workload
    (16, 3001, "poisson", 21, 3, 64, 4),      # blocks of unequal size, fluctuating R_i
    (32, 500, "nearest", 11, 2, 7, 5),
])
def test_analysis_side_by_side(L, R, kind, nT, theta, n_blocks, every):
    gpu = _pa(L, R, seed=5, resample=kind)
    ref = oracle.PA(L, R, 5, kind=oracle.POISSON if kind == "poisson" else oracle.NEAREST,
                    capacity=gpu.capacity)
    ref.init()
    assert_analysis_close(gpu.analyze(n_blocks), ref.analysis(n_blocks), "init")
    for i in range(1, nT):
        beta = i / (nT - 1)
        gpu.resample(beta)
        ref.resample(beta)
        gpu.anneal_step(theta)
        ref.sweep(theta)
        if i % every == 0 or i == nT - 1:
            assert np.array_equal(gpu.hashes(), ref.hashes())
            assert_analysis_close(gpu.analyze(n_blocks), ref.analysis(n_blocks), f"step {i}")


def test_analysis_full_size_L64_R1e6():
    """Full-size population (L = 64, R = 10^6, two steps of beta = i/300): the oracle analyses
    the device's own level, magnetisation and family arrays."""
    L, R = 64, 1_000_000
    N = L * L
    gpu = _pa(L, R, seed=7)
    for i in (1, 2):
        gpu.resample(i / 300)
        gpu.anneal_step(10)
    lv, mg, fm = gpu.replicas()
    E = 4 * lv.astype(np.int64) - 2 * N
    o = oracle.analysis(N, 2 / 300, E.astype(np.int32), mg, fm, 100)
    assert_analysis_close(gpu.analyze(100), o, "L=64 R=1e6")


def test_analysis_argument_errors_leave_context_usable():
    from paper_2102_06611_gb300 import PAError
    gpu = _pa(8, 50, seed=1)
    for bad in (1, 51, 2000):
        with pytest.raises(PAError):
            gpu.analyze(bad)
    r = gpu.analyze(50)   # blocks of one replica each
    assert r["n_blocks"] == 50 and r["families"] == 50
    assert r["var_mean_E_jack"] == pytest.approx(r["var_E"] / 50, rel=1e-12)
