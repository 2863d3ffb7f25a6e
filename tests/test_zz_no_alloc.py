"""tarang_diag_noalloc: the diagnostics entry point for callers that cannot
allocate device memory (its scratch is a static device array inside the
library).  Its output must equal tarang_diag's on the same state, on two
calls in a row (the second call reuses the scratch the first one left behind).

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import synth
from gpu_helpers import stream, sync, to_dev_c64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fk():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_07801_gb300 import build as b

    b.build()
    import paper_1805_07801_gb300 as m

    return m


def _kmax(n):
    return int(np.floor(np.sqrt(3.0) * (n // 2) + 0.5)) + 1


def _state(oracle_mod, n):
    if n <= 64:
        return oracle_mod.ic_random(synth.normal_fields(9, 3, (n, n, n)), k0=3.0, E0=0.5).astype(np.complex64)
    # larger grids: seeded complex values on every mode (the reduction does not
    # need a physical state, and this avoids the oracle's initial-field cost)
    hs = (n, n, n // 2 + 1)
    u = np.empty((3,) + hs, dtype=np.complex64)
    for c in range(3):
        u[c].real = synth.uniform_pm1(9, 2 * c, hs)
        u[c].imag = synth.uniform_pm1(9, 2 * c + 1, hs)
    return u


# n = 512 runs with the block count capped by the scratch's size (586 blocks
# of partials instead of 1216); 32 and 64 use the uncapped count
@pytest.mark.parametrize("n", [64, 32, 512])
def test_noalloc_diag_equals_tarang_diag_twice(fk, oracle_mod, n):
    import torch

    u = _state(oracle_mod, n)
    ud = to_dev_c64(u)
    del u
    plan = fk.fftk_plan_create(n, n, n)
    try:
        want_E, want_eps, want_EK = fk.tarang_diag(plan, ud.data_ptr(), 1e-3, stream())
    finally:
        fk.fftk_plan_destroy(plan)
    width = 2 + _kmax(n) + 1
    assert len(want_EK) == width - 2
    for _ in range(2):
        out = torch.full((width,), float("nan"), dtype=torch.float64, device="cuda:0")
        fk.tarang_diag_noalloc(n, ud.data_ptr(), 1e-3, out.data_ptr(), stream())
        sync()
        got = out.cpu().numpy()
        # same kernels, block count and summation order: equal to the last bit
        assert got[0] == want_E and got[1] == want_eps
        assert np.array_equal(got[2:], np.asarray(want_EK))
        assert abs(got[0] - want_E) <= 1e-13
        assert abs(got[1] - want_eps) <= 1e-13
        assert np.max(np.abs(got[2:] - np.asarray(want_EK))) <= 1e-14


def test_noalloc_diag_rejects_sizes_beyond_its_scratch(fk):
    import torch

    buf = torch.zeros(16, dtype=torch.float64, device="cuda:0")
    u = torch.zeros(64, dtype=torch.float32, device="cuda:0")
    with pytest.raises(fk.FFTKError) as e:
        fk.tarang_diag_noalloc(2048, u.data_ptr(), 1e-3, buf.data_ptr(), stream())
    assert e.value.status == fk.FFTK_ERR_UNSUPPORTED_SIZE
    with pytest.raises(fk.FFTKError) as e:
        fk.tarang_diag_noalloc(48, u.data_ptr(), 1e-3, buf.data_ptr(), stream())
    assert e.value.status == fk.FFTK_ERR_UNSUPPORTED_SIZE
