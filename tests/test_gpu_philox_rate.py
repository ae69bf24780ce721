"""The Philox measurement kernel (pa_philox_xor) computes the generator exactly as the sweep
does: its per-thread XOR of the four output words matches the oracle's Philox4x32-10 (itself
pinned to the published known-answer vectors) for a ragged thread count."""
import ctypes

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run(seed, n, calls):
    from paper_2102_06611_gb300 import _lib
    out = torch.full((n,), 0xDEAD, dtype=torch.int32, device="cuda")
    st = _lib.lib().pa_philox_xor(seed, n, calls, ctypes.c_void_p(out.data_ptr()), None)
    assert st == _lib.PA_OK
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("seed,n,calls", [(7, 300, 5), (0xFEEDFACECAFEBEEF, 37, 2), (1, 1, 0)])
def test_philox_xor_matches_oracle(seed, n, calls):
    got = _run(seed, n, calls)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for t in range(n):
        acc = 0
        for i in range(calls):
            x = oracle.philox4x32_10([i, t, 15 << 28, 0], key)
            acc ^= int(x[0]) ^ int(x[1]) ^ int(x[2]) ^ int(x[3])
        assert int(got[t]) == acc, (t, int(got[t]), acc)
