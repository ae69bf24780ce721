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


def test_tampered_checkpoint_is_rejected_before_the_device():
    """pa_load checks a checkpoint on the host: a state block that disagrees with the header
    or carries an error, an energy level, magnetisation, family id or copy number out of range
    each give PA_ERR_INVALID_ARG, and the context still loads the intact file afterwards."""
    import ctypes
    from paper_2102_06611_gb300 import PAError, _lib

    class Header(ctypes.Structure):   # the checkpoint header as pa_api.cu writes it
        _fields_ = [("magic", ctypes.c_ulonglong), ("cfg", _lib.pa_config),
                    ("step", ctypes.c_longlong), ("R_cur", ctypes.c_longlong), ("R_prev", ctypes.c_longlong),
                    ("n_log", ctypes.c_longlong), ("beta", ctypes.c_double), ("dbeta", ctypes.c_double),
                    ("i4", ctypes.c_int * 4)]

    L, R = 8, 300
    N = L * L
    a = _pa(L, R, 2)
    for i in (1, 2):
        a.resample(0.1 * i)
        a.anneal_step(2)
    ckpt = a.save()
    h = Header.from_buffer_copy(ckpt[:ctypes.sizeof(Header)])
    R_cur, R_prev, n_log = h.R_cur, h.R_prev, h.n_log
    H = ctypes.sizeof(Header)
    end_counts = len(ckpt) - n_log * ctypes.sizeof(_lib.pa_sched_entry)
    off_counts = end_counts - 4 * R_prev
    off_snap = off_counts - 4 * R_cur
    off_fam = off_snap - 4 * R_cur
    off_mag = off_fam - 4 * R_cur
    off_level = off_mag - 4 * R_cur
    assert np.frombuffer(ckpt[off_level:off_mag], np.int32).max() <= N

    def patched(off, fmt_value):
        b = bytearray(ckpt)
        b[off:off + len(fmt_value)] = fmt_value
        return bytes(b)

    i32 = lambda v: np.int32(v).tobytes()
    i64 = lambda v: np.int64(v).tobytes()
    bad = [patched(off_level + 4 * 7, i32(N + 1)),            # level above N
           patched(off_snap, i32(-1)),                          # step-start level below 0
           patched(off_mag + 4 * 3, i32(N + 2)),                # |M| > N
           patched(off_fam + 4 * (R_cur - 1), i32(-1)),         # family id out of range and order
           patched(off_counts, i32(-5)),                        # negative copy number
           patched(H, i64(R_cur + 1)),                          # state R_cur differs from the header
           patched(H + 44, i32(3))]                             # state block carries an error
    b = _pa(L, R, 2)
    for data in bad:
        with pytest.raises(PAError):
            b.load(data)
    b.load(ckpt)
    a.anneal_step(3)
    b.anneal_step(3)
    assert np.array_equal(a.hashes(), b.hashes())
