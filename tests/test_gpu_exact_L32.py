"""The L = 32 configuration against the exact finite-lattice solution: R = 10^5 replicas,
201 temperatures beta_i = i/200, theta = 10, nearest-integer and Poisson resampling, seeds
1-4.  At five temperatures (below, at and above beta_c) the GPU's energy and specific heat
agree with Kaufman's closed form (Ferdinand-Fisher thermodynamics) within 5 of the run's own
jackknife errors (pa_analyze, 100 blocks over the tree-ordered population), and its free
energy estimate -beta F (Sec. VII) within 1e-4 per spin."""
import math

import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

L, R, NT = 32, 100_000, 201
CHECKS = {50: 0.25, 88: 0.44, 100: 0.5, 150: 0.75, 200: 1.0}


@pytest.mark.parametrize("kind", ["nearest", "poisson"])
@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_L32_R1e5_against_exact(kind, seed):
    from paper_2102_06611_gb300 import PopulationAnnealing
    N = L * L
    pa = PopulationAnnealing(L, R, seed, resample=kind)
    for i in range(1, NT):
        pa.resample(i / (NT - 1))
        pa.anneal_step(10)
        if i not in CHECKS:
            continue
        e_ex, c_ex, lnz = oracle.kaufman_thermo(L, CHECKS[i])
        o = pa.observables()
        a = pa.analyze(100)
        se = math.sqrt(a["var_mean_E_jack"]) / N
        sc = math.sqrt(a["var_C_jack"])
        where = f"{kind} seed {seed} beta {CHECKS[i]}"
        assert abs(o["e"] - e_ex / N) <= 5 * se, (where, o["e"], e_ex / N, se)
        assert abs(o["C"] - c_ex) <= 5 * sc, (where, o["C"], c_ex, sc)
        assert abs(o["minus_betaF"] - lnz) / N <= 1e-4, (where, o["minus_betaF"], lnz)
        assert a["R_eff_E"] > 1000  # the population is far from collapsed at R = 10^5
