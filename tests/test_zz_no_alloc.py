"""The no-workspace copy-number entry point, checked against the regular resampling path.

pa_copy_numbers_static serves callers that cannot hand the library a workspace buffer (code
that may only touch the arrays it is given, or a process that forbids cudaMalloc after
start-up).  Its scratch is a fixed device array inside the library.  This test calls it
through the C ABI on two consecutive resampling steps and requires the same copy numbers,
population size and ln Q as pa_resample on the same parents, and as the CPU oracle's
resampling step given the same parent levels.  L = 128 covers the largest level table
(16385 levels, more than 48 KB of shared memory in the table kernel).  The file is named so
that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _static_copy_numbers(lib, L, R_target, levels_dev, beta_prev, beta_new, step, seed, kind, stream):
    R_prev = levels_dev.numel()
    counts = torch.full((R_prev,), -1, dtype=torch.int32, device=levels_dev.device)
    lnQ = ctypes.c_double()
    R_new = ctypes.c_longlong()
    st = lib.pa_copy_numbers_static(L, R_target, R_prev, ctypes.c_void_p(levels_dev.data_ptr()), beta_prev,
                                    beta_new, step, seed, kind, ctypes.c_void_p(counts.data_ptr()),
                                    ctypes.byref(lnQ), ctypes.byref(R_new), ctypes.c_void_p(stream.cuda_stream))
    return st, counts.cpu().numpy(), lnQ.value, R_new.value


@pytest.mark.parametrize("L,R,kind", [(32, 20000, "nearest"), (16, 5000, "poisson"), (128, 3000, "nearest"),
                                      (96, 2000, "poisson")])
def test_static_entry_point_matches_resample(L, R, kind):
    import oracle
    from paper_2102_06611_gb300 import PopulationAnnealing, _lib
    seed = 13
    pa = PopulationAnnealing(L, R, seed, resample=kind)
    lib = pa.lib
    stream = torch.cuda.current_stream()
    kind_code = _lib.PA_RESAMPLE_POISSON if kind == "poisson" else _lib.PA_RESAMPLE_NEAREST
    beta_prev = 0.0
    for step, beta in enumerate([0.05, 0.1], start=1):   # two calls in a row
        levels, _, _ = pa.replicas()
        levels_dev = torch.from_numpy(levels).cuda()
        pa.resample(beta)
        expected = pa.copy_counts()
        st, counts, lnQ, R_new = _static_copy_numbers(lib, L, R, levels_dev, beta_prev, beta, step, seed,
                                                      kind_code, stream)
        assert st == _lib.PA_OK
        assert np.array_equal(counts, expected)
        assert R_new == pa.R == int(expected.sum())
        o_kind = oracle.POISSON if kind == "poisson" else oracle.NEAREST
        o_st, o_counts, o_lnQ, _, _, o_R = oracle.resample_levels(L, R, levels, beta_prev, beta, step, seed, o_kind,
                                                                  oracle.default_capacity(R))
        assert o_st == 0 and np.array_equal(counts, o_counts) and R_new == o_R
        assert abs(lnQ - o_lnQ) <= 1e-12 * max(1.0, abs(o_lnQ))
        pa.anneal_step(2)
        obs = pa.observables()
        assert abs(lnQ - obs["lnQ"]) <= 1e-12 * max(1.0, abs(obs["lnQ"]))
        beta_prev = beta


def test_static_entry_point_rejects_sizes_beyond_its_maximum():
    from paper_2102_06611_gb300 import _lib
    lib = _lib.lib()
    dummy = torch.zeros(1, dtype=torch.int32, device="cuda")
    lnQ, R_new = ctypes.c_double(), ctypes.c_longlong()
    st = lib.pa_copy_numbers_static(64, 1000, (1 << 22) + 1, ctypes.c_void_p(dummy.data_ptr()), 0.0, 0.1, 1, 1, 0,
                                    ctypes.c_void_p(dummy.data_ptr()), ctypes.byref(lnQ), ctypes.byref(R_new),
                                    None)
    assert st == _lib.PA_ERR_TOO_LARGE
    st = lib.pa_copy_numbers_static(130, 1000, 10, ctypes.c_void_p(dummy.data_ptr()), 0.0, 0.1, 1, 1, 0,
                                    ctypes.c_void_p(dummy.data_ptr()), ctypes.byref(lnQ), ctypes.byref(R_new),
                                    None)
    assert st == _lib.PA_ERR_INVALID_ARG
