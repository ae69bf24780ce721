"""Checkpoint / resume: a run saved at step k and resumed in a fresh context ends bit-identical
to the uninterrupted run (counter-based random numbers carry no generator state)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pa(*a, **k):
    from paper_2102_06611_gb300 import PopulationAnnealing
    return PopulationAnnealing(*a, **k)


@pytest.mark.parametrize("L,R,kind", [(16, 1500, "nearest"), (32, 800, "poisson")])
def test_resume_is_bit_identical(L, R, kind):
    seed, nT, theta = 4, 9, 3
    full = _pa(L, R, seed, resample=kind)
    for i in range(1, nT):
        full.resample(i / (nT - 1))
        full.anneal_step(theta)
    first = _pa(L, R, seed, resample=kind)
    for i in range(1, 5):
        first.resample(i / (nT - 1))
        first.anneal_step(theta)
    ckpt = first.save()
    first.close()
    resumed = _pa(L, R, seed, resample=kind)
    resumed.load(ckpt)
    for i in range(5, nT):
        resumed.resample(i / (nT - 1))
        resumed.anneal_step(theta)
    assert np.array_equal(resumed.hashes(), full.hashes())
    assert resumed.observables() == full.observables()
    assert [e["beta"] for e in resumed.schedule_log()] == [e["beta"] for e in full.schedule_log()]


def test_checkpoint_mid_step_and_rejections():
    from paper_2102_06611_gb300 import PAError
    a = _pa(8, 400, 1)
    a.resample(0.3)
    a.anneal_step(2)          # save between two sweep calls of one temperature
    ckpt = a.save()
    a.anneal_step(3)
    b = _pa(8, 400, 1)
    b.load(ckpt)
    b.anneal_step(3)
    assert np.array_equal(a.hashes(), b.hashes()) and a.decorrelation() == b.decorrelation()
    other = _pa(8, 400, 2)    # different seed: a different configuration
    with pytest.raises(PAError):
        other.load(ckpt)
    with pytest.raises(PAError):
        b.load(ckpt[:100])
