"""Degenerate and ragged cases of the CUDA path against the oracle: a population of one
replica, extinction under Poisson resampling, a single enormous temperature step, and
population sizes that leave ragged warps, blocks and tie queues."""
import numpy as np
import pytest

import oracle
from side_by_side import run_side_by_side

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pa(*a, **k):
    from paper_2102_06611_gb300 import PopulationAnnealing
    return PopulationAnnealing(*a, **k)


@pytest.mark.parametrize("L", [4, 16, 64, 128])
def test_single_replica_population(L):
    """R = 1 with nearest-integer copies: tau_hat = 1 exactly, so the population stays one
    replica; every step matches the oracle."""
    gpu = _pa(L, 1, seed=3)
    ref = oracle.PA(L, 1, 3, capacity=gpu.capacity)
    run_side_by_side(gpu, ref, [i / 8 for i in range(1, 9)], 2)
    assert gpu.R == 1


def test_poisson_extinction_is_a_clean_error():
    """Poisson copies of a single replica (mean 1) die out with probability 1/e per step: the
    device reports the empty population (PA_ERR_NUMERIC) at the same step as the oracle,
    without a fault, and the context refuses further work."""
    from paper_2102_06611_gb300 import PAError
    gpu = _pa(8, 1, seed=2, resample="poisson")
    ref = oracle.PA(8, 1, 2, kind=oracle.POISSON, capacity=gpu.capacity)
    ref.init()
    step = None
    for i in range(1, 40):
        st = ref.resample(i / 40)
        gpu.resample(i / 40)
        if st != 0:
            step = i
            assert st == 6
            with pytest.raises(PAError) as ei:
                gpu.sync()
            assert ei.value.status == 6
            break
        gpu.anneal_step(1)
        ref.sweep(1)
        assert np.array_equal(gpu.hashes(), ref.hashes())
    assert step is not None
    with pytest.raises(PAError):
        gpu.anneal_step(1)


@pytest.mark.parametrize("kind", ["nearest", "poisson", "multinomial"])
def test_one_enormous_temperature_step(kind):
    """beta 0 -> 20 in one step: every weight but the lowest occupied level's underflows to
    (nearly) zero; copies, ln Q and the swept population still match the oracle."""
    k = {"nearest": oracle.NEAREST, "poisson": oracle.POISSON, "multinomial": oracle.MULTINOMIAL}[kind]
    gpu = _pa(8, 1000, seed=5, resample=kind)
    ref = oracle.PA(8, 1000, 5, kind=k, capacity=gpu.capacity)
    run_side_by_side(gpu, ref, [20.0, 20.0, 21.5], 3)


@pytest.mark.parametrize("L,R", [(8, 31), (8, 33), (32, 1023), (32, 1025), (64, 3), (64, 4097), (128, 5)])
def test_ragged_population_sizes(L, R):
    gpu = _pa(L, R, seed=9)
    ref = oracle.PA(L, R, 9, capacity=gpu.capacity)
    run_side_by_side(gpu, ref, [0.3, 0.6, 0.9], 2)
