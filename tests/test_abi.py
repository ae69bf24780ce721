"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every symbol
that include/pa.h declares.  No compute call is made here."""
import ctypes
import os
import re

import pytest

from paper_2102_06611_gb300 import _lib
from paper_2102_06611_gb300 import build as pabuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def declared_symbols():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(pa_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_method_steps():
    names = declared_symbols()
    for n in ("pa_init", "pa_resample", "pa_anneal_step", "pa_observables"):
        assert n in names


def test_library_builds_and_exports_every_declared_symbol():
    path = pabuild.build()
    lib = ctypes.CDLL(path)
    for n in declared_symbols():
        assert hasattr(lib, n), n
    # the Python binding declares exactly the header's entry points
    assert set(_lib.SIGNATURES) == set(declared_symbols())


def test_query_sizes_is_host_only():
    lib = _lib.lib()
    cfg = _lib.pa_config(L=64, resample=0, R=1000, capacity=2000, seed=7)
    sz = _lib.pa_sizes()
    assert lib.pa_query_sizes(ctypes.byref(cfg), ctypes.byref(sz)) == _lib.PA_OK
    assert sz.bytes_per_replica == 512
    assert sz.spin_bytes == 512 * 2000 and sz.int_bytes == 4 * 2000
    assert sz.work_bytes > 0 and sz.work_bytes % 256 == 0
    cfg128 = _lib.pa_config(L=128, resample=0, R=10, capacity=10, seed=1)
    assert lib.pa_query_sizes(ctypes.byref(cfg128), ctypes.byref(sz)) == _lib.PA_OK
    assert sz.bytes_per_replica == 2048
    hb = _lib.pa_config(L=16, resample=1, R=10, capacity=30, seed=1, update=_lib.PA_UPDATE_HEATBATH)
    assert lib.pa_query_sizes(ctypes.byref(hb), ctypes.byref(sz)) == _lib.PA_OK


@pytest.mark.parametrize("L,bpr", [(6, 48), (20, 160), (66, 1056), (126, 2016)])
def test_query_sizes_any_even_L(L, bpr):
    """Every even 4 <= L <= 128 is accepted; a replica is L rows of two half-row words
    (32-bit for L <= 64, 64-bit above)."""
    cfg = _lib.pa_config(L=L, resample=0, R=10, capacity=20, seed=1)
    sz = _lib.pa_sizes()
    assert _lib.lib().pa_query_sizes(ctypes.byref(cfg), ctypes.byref(sz)) == _lib.PA_OK
    assert sz.bytes_per_replica == bpr


def test_philox_rate_rejects_bad_arguments():
    lib = _lib.lib()
    assert lib.pa_philox_xor(1, 0, 4, ctypes.c_void_p(256), None) == _lib.PA_ERR_INVALID_ARG
    assert lib.pa_philox_xor(1, 10, -1, ctypes.c_void_p(256), None) == _lib.PA_ERR_INVALID_ARG
    assert lib.pa_philox_xor(1, 10, 4, None, None) == _lib.PA_ERR_INVALID_ARG


def test_batches_take_every_even_size():
    """Batches take every even 4 <= L <= 128 (register kernels or the shared-memory sweep) and
    reject the sizes a single run rejects."""
    lib = _lib.lib()
    n = ctypes.c_size_t()
    for L, st in ((16, _lib.PA_OK), (20, _lib.PA_OK), (100, _lib.PA_OK), (6, _lib.PA_OK), (7, _lib.PA_ERR_INVALID_ARG),
                  (2, _lib.PA_ERR_INVALID_ARG), (130, _lib.PA_ERR_INVALID_ARG)):
        d = (_lib.pa_run_desc * 1)(_lib.pa_run_desc(_lib.pa_config(L=L, resample=0, R=100, capacity=200, seed=1),
                                                    5, 1))
        assert lib.pa_batch_query_sizes(1, d, ctypes.byref(n)) == st


@pytest.mark.parametrize("bad", [dict(L=2), dict(L=7), dict(L=130), dict(L=256), dict(R=0), dict(capacity=5, R=10),
                                 dict(resample=3), dict(capacity=2 ** 31), dict(update=2), dict(pad=1)])
def test_query_sizes_rejects_bad_configs(bad):
    args = dict(L=8, resample=0, R=10, capacity=20, seed=1)
    args.update(bad)
    cfg = _lib.pa_config(**args)
    sz = _lib.pa_sizes()
    assert _lib.lib().pa_query_sizes(ctypes.byref(cfg), ctypes.byref(sz)) == _lib.PA_ERR_INVALID_ARG


def test_init_rejects_null_and_misaligned_buffers():
    lib = _lib.lib()
    cfg = _lib.pa_config(L=8, resample=0, R=10, capacity=20, seed=1)
    bufs = _lib.pa_buffers()
    ctx = ctypes.c_void_p()
    assert lib.pa_init(ctypes.byref(cfg), ctypes.byref(bufs), None, ctypes.byref(ctx)) == _lib.PA_ERR_INVALID_ARG
    for b in range(2):
        bufs.spins[b] = bufs.level[b] = bufs.mag[b] = bufs.fam[b] = 256 * (b + 1) + 4
    bufs.work = 4096
    assert lib.pa_init(ctypes.byref(cfg), ctypes.byref(bufs), None, ctypes.byref(ctx)) == _lib.PA_ERR_INVALID_ARG
    assert not ctx.value


def test_no_cpu_fallback_without_a_gpu():
    """Without a CUDA device the product path raises instead of computing anywhere else."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2102_06611_gb300 import PopulationAnnealing
    with pytest.raises(Exception):
        PopulationAnnealing(8, 100, 1)
