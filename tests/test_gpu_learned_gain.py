"""What the trained schedule network gains over the plain adaptive schedule: the same anneal
(beta 0 -> 1) in less wall time and with fewer sweeps, with the free energy per spin still
within 1e-4 of the exact finite-lattice value (Kaufman, tests/golden/exact_lnZ.json).  The
ablation arm "rule" (bisection for dbeta, the measured-decorrelation rule for theta, no
network) must reach the same accuracy; its wall time against the learned arm is reported by
the benchmark."""
import json
import os

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "exact_lnZ.json")


def test_trained_schedule_beats_plain_at_equal_accuracy():
    from paper_2102_06611_gb300 import PopulationAnnealing
    from paper_2102_06611_gb300.learned import ScheduleMLP, anneal
    from paper_2102_06611_gb300.train_schedule import DEFAULT_WEIGHTS

    L, R, seed = 64, 50_000, 3
    exact = json.load(open(GOLDEN))["lnZ"][str(L)]["1.0"]
    model = ScheduleMLP.load(DEFAULT_WEIGHTS)
    res = {}
    for mode in ("plain", "learned", "rule", "plain"):  # plain twice: the first run warms up
        pa = PopulationAnnealing(L, R, seed)
        res[mode] = anneal(pa, mode, model)
        pa.close()
    for mode, r in res.items():
        assert r["beta"] == 1.0
        assert abs(r["minus_betaF"] - exact) / (L * L) <= 1e-4, (mode, r)
    assert res["learned"]["sweeps"] < 0.6 * res["plain"]["sweeps"]
    # the ablation without the network (bisection + the decorrelation rule for theta) also
    # needs far fewer sweeps than theta = 10 everywhere
    assert res["rule"]["sweeps"] < 0.6 * res["plain"]["sweeps"]
    assert res["learned"]["wall_s"] < res["plain"]["wall_s"]
    assert res["learned"]["fallbacks"] <= res["learned"]["steps"] // 10
