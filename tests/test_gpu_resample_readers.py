"""Readers of a population right after pa_resample (Sec. II step 2): hashes, spin export, a
sweep count of 0, a checkpoint taken before the step's first sweep, and a second resampling
with no sweep in between (which must measure the children first: Eqs. Q and taus use the
parents' histogram).  Every path gives the same population, hash for hash, as the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402


def _pa(L, R, seed, update="metropolis"):
    from paper_2102_06611_gb300 import PopulationAnnealing
    return PopulationAnnealing(L, R, seed, update=update)


@pytest.mark.parametrize("L,R,update", [(16, 3000, "metropolis"), (64, 2000, "metropolis"),
                                        (64, 2000, "heatbath"), (10, 2000, "metropolis")])
def test_every_reader_sees_the_children(L, R, update):
    """Resample then sweep, against: hashes right after the resampling, an export of the
    spins, a sweep count of 0 before the sweeps, a checkpoint taken between resampling and
    sweep (its step-start levels are not written yet); the post-resampling hashes against the
    oracle's."""
    seed, theta = 5, 3
    betas = [0.1, 0.3, 0.5, 0.8]
    fused, early, zero, ck = (_pa(L, R, seed, update) for _ in range(4))
    ref = oracle.PA(L, R, seed, kind=oracle.NEAREST,
                    update=oracle.HEATBATH if update == "heatbath" else oracle.METROPOLIS)
    ref.init()
    for b in betas:
        for p in (fused, early, zero, ck):
            p.resample(b)
        assert ref.resample(b) == 0
        h_early = early.hashes()
        assert np.array_equal(h_early, ref.hashes())
        words = zero.export_spins(0, 3)
        assert words.shape[0] == 3
        zero.anneal_step(0)                           # measure only, then the sweeps
        blob = ck.save()                              # a checkpoint holds the children's spins
        ck.load(blob)
        fused.anneal_step(theta)
        early.anneal_step(theta)
        zero.anneal_step(theta)
        ck.anneal_step(theta)
        ref.sweep(theta)
        want = ref.hashes()
        for p in (fused, early, zero, ck):
            assert np.array_equal(p.hashes(), want)
            assert np.array_equal(p.histogram(), fused.histogram())
        assert fused.observables() == early.observables()
    for p in (fused, early, zero, ck):
        p.close()


def test_two_resamplings_in_a_row():
    """A resampling right after another (no sweep in between) draws from the children's own
    histogram, as the oracle does."""
    L, R, seed = 32, 2500, 8
    pa = _pa(L, R, seed)
    ref = oracle.PA(L, R, seed)
    ref.init()
    for b in (0.02, 0.05):
        pa.resample(b)
        assert ref.resample(b) == 0
    pa.anneal_step(2)
    ref.sweep(2)
    assert np.array_equal(pa.hashes(), ref.hashes())
    assert np.array_equal(pa.copy_counts(), ref.counts())
    pa.close()
