"""Weighted averages over independent runs (Sec. VIII) on the GPU: a batch of runs that
differ only in their seed is recorded at every temperature step, and pa_weighted_average
is compared with the oracle's formula applied to the same records; each run's size factor
sum_k ln(R_{k-1}/R) is covered by the single-run parity tests."""
import ctypes

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ["M_eff", "max_weight", "var_minus_betaF", "minus_betaF_combined", "e", "C", "m", "m2", "chi",
        "e_plain", "C_plain", "m_plain", "m2_plain", "chi_plain"]


def _host_records(rec_dev):
    from paper_2102_06611_gb300 import OBS_BYTES, pa_obs
    raw = rec_dev.cpu().numpy().tobytes()
    M = len(raw) // OBS_BYTES
    return [pa_obs.from_buffer_copy(raw[i * OBS_BYTES:(i + 1) * OBS_BYTES]) for i in range(M)]


def _oracle_weighted(recs, mode):
    return oracle.weighted_average([r.R for r in recs], [r.R_target for r in recs], [r.minus_betaF for r in recs],
                                   [r.sum_lnRratio for r in recs], [[r.e, r.C, r.m, r.m2, r.chi] for r in recs],
                                   mode)


@pytest.mark.parametrize("resample", ["nearest", "poisson"])
def test_weighted_average_matches_oracle(resample):
    from paper_2102_06611_gb300 import OBS_BYTES, weighted_average
    from paper_2102_06611_gb300.batch import Batch, RunSpec
    M, steps = 12, 20
    runs = [RunSpec(L=8, R=800, seed=11 + m, n_temps=steps + 1, theta=5, resample=resample) for m in range(M)]
    b = Batch(runs)
    words = OBS_BYTES // 8
    rec = torch.zeros((steps, M, words), dtype=torch.int64, device="cuda")
    for s in range(steps):
        b.step()
        b.record(rec[s])
    torch.cuda.synchronize()
    for s in (0, 4, 9, 19):
        recs = _host_records(rec[s])
        assert all(r.step == s + 1 for r in recs)
        for mode_name, mode in (("standard", 0), ("modified", 1)):
            g = weighted_average(rec[s], mode_name)
            o = _oracle_weighted(recs, mode)
            assert g["status"] == 0 and g["M"] == M and g["step"] == s + 1
            for k in KEYS:
                assert abs(g[k] - o[k]) <= 1e-12 * max(1.0, abs(o[k])), f"step {s + 1} {mode_name} {k}"
    # at beta = 1 the weights are far from uniform only if sigma^2(beta F) is large
    g = weighted_average(rec[steps - 1])
    assert 1.0 <= g["M_eff"] <= M
    b.close()


def test_weighted_average_rejects_mixed_steps():
    from paper_2102_06611_gb300 import OBS_BYTES, PopulationAnnealing, weighted_average
    a = PopulationAnnealing(8, 100, 1)
    c = PopulationAnnealing(8, 100, 2)
    rec = torch.zeros((2, OBS_BYTES // 8), dtype=torch.int64, device="cuda")
    a.resample(0.1)
    a.anneal_step(1)
    c.anneal_step(1)
    a.record(rec[0])
    c.record(rec[1])
    g = weighted_average(rec)
    assert g["status"] == 1   # PA_ERR_INVALID_ARG: records of different temperature steps
