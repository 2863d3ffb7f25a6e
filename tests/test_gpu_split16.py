"""FFTK_R32_SPLIT16: the y and x passes' radix-16 stages on the tensor cores
(tcgen05) with split FP16 hi/lo operands and FP32 accumulation.

Tolerance: relative L2 <= 1e-5 against the FP64 oracle.  Each
tensor-core stage drops only x_lo * W_lo (2^-22 relative) and rounds the FP32
accumulation; four such stages per pair plus the FP32 stages stay well below.
"""
import numpy as np
import pytest

import synth
from gpu_helpers import empty_c64, empty_real, from_dev_c64, rel_l2, stream, sync, to_dev_c64, to_dev_real

pytestmark = pytest.mark.gpu

REL = 1e-5


@pytest.fixture(scope="module")
def fk():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_07801_gb300 import build as b

    b.build()
    import paper_1805_07801_gb300 as m

    return m


def _plan(fk, shape):
    return fk.fftk_plan_create(*shape, fk.FFTK_R32_SPLIT16)


SHAPES = [
    (256, 4, 8), (16, 256, 4), (512, 8, 16), (4, 512, 32), (1024, 4, 4), (8, 1024, 2),
    (2048, 2, 4), (2, 2048, 8), (256, 256, 16), (64, 512, 64), (512, 64, 8), (128, 64, 32),
]


@pytest.mark.parametrize("shape", SHAPES)
def test_split16_r2c_and_c2r_match_oracle(fk, oracle_mod, shape):
    f = synth.uniform_pm1(4, 0, shape)
    hs = (shape[0], shape[1], shape[2] // 2 + 1)
    plan = _plan(fk, shape)
    try:
        x = to_dev_real(f)
        F = empty_c64(hs)
        fk.fftk_r2c(plan, x.data_ptr(), F.data_ptr(), 1, stream())
        fk.fftk_sync(plan, stream())
        Fg = from_dev_c64(F)
        Fo = oracle_mod.rfft3(f.astype(np.float64))
        assert rel_l2(Fg, Fo) < REL
        Fin = Fo.astype(np.complex64)
        y = empty_real(shape)
        Fd = to_dev_c64(Fin)
        fk.fftk_c2r(plan, Fd.data_ptr(), y.data_ptr(), 1, stream())
        fk.fftk_sync(plan, stream())
        go = oracle_mod.irfft3(Fin.astype(np.complex128), shape[2])
        assert rel_l2(y.cpu().numpy(), go) < REL
    finally:
        fk.fftk_plan_destroy(plan)


def test_split16_batched_deterministic_and_scaled_inputs(fk, oracle_mod):
    # widely different magnitudes across the batch: the power-of-two scaling
    # keeps every element inside the FP16 range
    shape, B = (256, 16, 32), 3
    f = np.stack([synth.uniform_pm1(5, b, shape) * s for b, s in enumerate([1e-6, 1.0, 3e4])]).astype(np.float32)
    plan = _plan(fk, shape)
    try:
        x = to_dev_real(f)
        F1 = empty_c64((B,) + shape[:2] + (shape[2] // 2 + 1,))
        F2 = empty_c64((B,) + shape[:2] + (shape[2] // 2 + 1,))
        fk.fftk_r2c(plan, x.data_ptr(), F1.data_ptr(), B, stream())
        fk.fftk_r2c(plan, x.data_ptr(), F2.data_ptr(), B, stream())
        fk.fftk_sync(plan, stream())
        import torch

        assert torch.equal(F1, F2)
        Fg = from_dev_c64(F1)
    finally:
        fk.fftk_plan_destroy(plan)
    for b in range(B):
        Fo = oracle_mod.rfft3(f[b].astype(np.float64))
        assert rel_l2(Fg[b], Fo) < REL


def test_split16_full_size_1024_pair(fk, oracle_mod):
    """1024^3 in the benchmark's configuration: round trip and sampled
    coefficients by direct O(N^3) sums."""
    import torch

    n = 1024
    shape = (n, n, n)
    plan = _plan(fk, shape)
    try:
        x = torch.empty(shape, dtype=torch.float32, device="cuda:0")
        fk.fftk_fill_normal(x.data_ptr(), x.numel(), 0, 0, stream())
        F = empty_c64((n, n, n // 2 + 1))
        y = empty_real(shape)
        fk.fftk_r2c(plan, x.data_ptr(), F.data_ptr(), 1, stream())
        fk.fftk_c2r(plan, F.data_ptr(), y.data_ptr(), 1, stream())
        fk.fftk_sync(plan, stream())
        rt = (torch.linalg.vector_norm((y - x).double()) / torch.linalg.vector_norm(x.double())).item()
        assert rt < REL
        f = x.cpu().numpy()
        del y
        Fh = from_dev_c64(F)
    finally:
        fk.fftk_plan_destroy(plan)
    rms = float(np.sqrt(np.mean(np.abs(Fh) ** 2)))
    for (a, b, c) in [(0, 0, 0), (3, 1000, 7), (512, 512, 512), (77, 5, 300)]:
        want = oracle_mod.rfft3_coeff(f, a, b, c)
        assert abs(Fh[a, b, c] - want) < 5e-5 * rms


def test_split16_tiny_and_mixed_magnitude_columns(fk, oracle_mod):
    """Columns whose values lie near FP32's smallest normals (and columns that
    mix 1 and 1e-38) keep a finite power-of-two scale: the transforms stay
    finite and within the split mode's error of the FP64 oracle."""
    shape = (256, 256, 8)
    f = synth.uniform_pm1(7, 0, shape).astype(np.float64)
    f[:, :, :4] *= 1e-38
    f[:128] *= 1e-30
    hs = (shape[0], shape[1], shape[2] // 2 + 1)
    plan = _plan(fk, shape)
    try:
        x = to_dev_real(f.astype(np.float32))
        F = empty_c64(hs)
        fk.fftk_r2c(plan, x.data_ptr(), F.data_ptr(), 1, stream())
        y = empty_real(shape)
        fk.fftk_c2r(plan, F.data_ptr(), y.data_ptr(), 1, stream())
        sync()
        Fg, yg = from_dev_c64(F), y.cpu().numpy()
    finally:
        fk.fftk_plan_destroy(plan)
    assert np.all(np.isfinite(Fg)) and np.all(np.isfinite(yg))
    Fo = oracle_mod.rfft3(f.astype(np.float32).astype(np.float64))
    assert rel_l2(Fg, Fo) < 1e-5
    assert rel_l2(yg, f.astype(np.float32)) < 1e-5
