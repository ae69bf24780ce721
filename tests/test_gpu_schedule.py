"""Adaptive temperature steps on the GPU vs the oracle: the proposed beta and its overlap
must agree bit for bit, and a whole adaptive anneal must stay in parity."""
import math

import numpy as np
import pytest

import oracle
from side_by_side import assert_obs_close, compare_population

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pa(*a, **k):
    from paper_2102_06611_gb300 import PopulationAnnealing
    return PopulationAnnealing(*a, **k)


@pytest.mark.parametrize("L,R,target", [(8, 1500, 0.8), (16, 2000, 0.8), (32, 800, 0.5), (20, 600, 0.8)])
def test_adaptive_anneal_parity(L, R, target):
    from paper_2102_06611_gb300 import _lib
    seed, theta, dmax, bf = 21, 3, 0.1, 1.0
    gpu = _pa(L, R, seed)
    ref = oracle.PA(L, R, seed, capacity=gpu.capacity)
    ref.init()
    betas = []
    beta = 0.0
    for i in range(1, 400):
        bg, ag = gpu.propose_schedule(target, dmax, bf)
        bo, ao = ref.propose_bisect(bf, dmax, target)
        assert bg == bo and ag == ao, (i, bg, bo, ag, ao)
        assert ag >= target or bg == bf
        gpu.resample(bg)
        assert ref.resample(bo) == 0
        gpu.anneal_step(theta)
        ref.sweep(theta)
        betas.append(bg)
        beta = bg
        if beta == bf:
            break
    assert beta == bf
    compare_population(gpu, ref, "end of adaptive anneal")
    assert_obs_close(gpu.observables(), ref.observables(), "end of adaptive anneal")
    log = gpu.schedule_log()
    assert [e["beta"] for e in log] == betas
    assert all(e["source"] == _lib.PA_SCHED_BISECT and e["theta"] == theta for e in log)
    assert all(e["alpha"] >= target for e in log[:-1])


def test_proposal_after_resampling_measures_first():
    L, R, seed = 16, 1000, 3
    gpu = _pa(L, R, seed)
    ref = oracle.PA(L, R, seed, capacity=gpu.capacity)
    ref.init()
    gpu.resample(0.2)
    ref.resample(0.2)
    bg, ag = gpu.propose_schedule(0.8, 0.1, 1.0)   # the population was not swept yet
    bo, ao = ref.propose_bisect(1.0, 0.1, 0.8)
    assert (bg, ag) == (bo, ao)
    gpu.resample(0.25)                              # a caller-chosen beta is logged as such
    log = gpu.schedule_log()
    assert [e["source"] for e in log] == [0, 0] and math.isnan(log[1]["alpha"])


def test_full_size_proposal_L64_R1e6():
    L, R, seed = 64, 1_000_000, 7
    gpu = _pa(L, R, seed)
    for beta in (0.0, 0.3):
        if beta > 0:
            gpu.resample(beta)
            gpu.anneal_step(10)
        h = gpu.histogram().astype(np.int64)
        bg, ag = gpu.propose_schedule(0.8, 0.1, 1.0)
        bo, ao = oracle.bisect_next_beta(L * L, h, beta, 1.0, 0.1, 0.8)
        assert (bg, ag) == (bo, ao)
        assert ag >= 0.8
