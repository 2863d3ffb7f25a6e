"""GPU parity of transforms on 3 * 2^m grids (the paper's 768^3, 1536^3 and
3072^3 sizes, Sec. 5): one radix-3 step over power-of-two sub-lines in the
z, y and x passes, against the FP64 oracle (lines of 3 * 2^m points by the
DFT's definition), through the C ABI.  Same bars as the power-of-two
transforms: relative L2 2e-6, 1e-5 of the largest coefficient per element.
"""
import numpy as np
import pytest

import synth
from gpu_helpers import from_dev_c64, rel_l2, stream, sync, to_dev_c64

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


def _pair(fk, shape, f, dtype=None, batch=1):
    import torch

    nx, ny, nz = shape
    plan = fk.fftk_plan_create(nx, ny, nz, dtype if dtype is not None else fk.FFTK_R32)
    try:
        x = torch.from_numpy(np.ascontiguousarray(f, dtype=np.float32)).to("cuda:0")
        F = torch.empty((batch, nx, ny, nz // 2 + 1, 2), dtype=torch.float32, device="cuda:0")
        y = torch.empty_like(x)
        fk.fftk_r2c(plan, x.data_ptr(), F.data_ptr(), batch, stream())
        fk.fftk_c2r(plan, F.data_ptr(), y.data_ptr(), batch, stream())
        sync()
        return from_dev_c64(F), y.cpu().numpy()
    finally:
        fk.fftk_plan_destroy(plan)


@pytest.mark.parametrize("shape", [(6, 12, 24), (12, 24, 48), (96, 48, 24), (24, 96, 12), (96, 96, 96),
                                   (768, 4, 12), (4, 1536, 12), (3072, 2, 12), (2, 2, 3072), (64, 48, 32)])
def test_r2c_c2r_match_oracle(fk, oracle_mod, shape):
    f = synth.uniform_pm1(31, 0, shape)
    F, y = _pair(fk, shape, f[None])
    want = oracle_mod.rfft3(f.astype(np.float64))
    assert rel_l2(F[0], want) < 2e-6
    assert np.max(np.abs(F[0] - want)) < 1e-5 * np.max(np.abs(want))
    # the unnormalised inverse of the normalised forward is the input
    assert rel_l2(y[0], f) < 2e-6


def test_inverse_of_oracle_spectrum(fk, oracle_mod):
    import torch

    shape = (48, 24, 96)
    f = synth.uniform_pm1(32, 0, shape).astype(np.float64)
    want = oracle_mod.rfft3(f)
    plan = fk.fftk_plan_create(*shape)
    try:
        Fd = to_dev_c64(want[None])
        y = torch.empty((1,) + shape, dtype=torch.float32, device="cuda:0")
        fk.fftk_c2r(plan, Fd.data_ptr(), y.data_ptr(), 1, stream())
        sync()
    finally:
        fk.fftk_plan_destroy(plan)
    assert rel_l2(y.cpu().numpy()[0], oracle_mod.irfft3(want, shape[2])) < 2e-6


def test_batched_and_split16_plan(fk, oracle_mod):
    shape = (24, 48, 12)
    f = np.stack([synth.uniform_pm1(33, i, shape) for i in range(2)])
    for dtype in (fk.FFTK_R32, fk.FFTK_R32_SPLIT16):
        F, _ = _pair(fk, shape, f, dtype=dtype, batch=2)
        for i in range(2):
            assert rel_l2(F[i], oracle_mod.rfft3(f[i].astype(np.float64))) < 2e-6


def test_full_size_768_sampled_coefficients(fk, oracle_mod):
    import torch

    n = 768
    dev = torch.device("cuda:0")
    plan = fk.fftk_plan_create(n, n, n)
    try:
        x = torch.empty((n, n, n), dtype=torch.float32, device=dev)
        fk.fftk_fill_uniform(x.data_ptr(), x.numel(), 34, 0, stream())
        F = torch.empty((n, n, n // 2 + 1, 2), dtype=torch.float32, device=dev)
        y = torch.empty_like(x)
        fk.fftk_r2c(plan, x.data_ptr(), F.data_ptr(), 1, stream())
        fk.fftk_c2r(plan, F.data_ptr(), y.data_ptr(), 1, stream())
        sync()
        err = float(torch.linalg.vector_norm(y.double() - x.double()) / torch.linalg.vector_norm(x.double()))
        xh = x.cpu().numpy()
        Fh = F.cpu().numpy()
    finally:
        fk.fftk_plan_destroy(plan)
    assert err < 2e-6
    rng = np.random.default_rng(1)
    picks = [(0, 0, 0), (n - 1, n - 1, n // 2), (1, 2, 3), (256, 512, 384)]
    picks += [(int(rng.integers(0, n)), int(rng.integers(0, n)), int(rng.integers(0, n // 2 + 1))) for _ in range(4)]
    scale = 1.0 / np.sqrt(3.0 * n**3)  # rms coefficient of uniform(-1, 1) input
    for a, b, c in picks:
        want = oracle_mod.rfft3_coeff(xh, a, b, c)
        got = complex(Fh[a, b, c, 0], Fh[a, b, c, 1])
        assert abs(got - want) < 1e-4 * scale, (a, b, c, got, want)


def test_radix3_grids_outside_the_solver_and_bases(fk):
    # the solver takes 3 * 2^m cubes up to 768 (tests/test_gpu_ns_radix3.py);
    # the sine/cosine bases and the learned closure need power-of-two axes
    import torch

    plan = fk.fftk_plan_create(48, 48, 48)
    try:
        u = torch.zeros((3, 48, 48, 25, 2), device="cuda:0")
        with pytest.raises(fk.FFTKError):
            fk.fftk_forward(plan, "SFF", u.data_ptr(), u.data_ptr() + 4 * 48**3, 1, stream())
        model = fk.make_sgs_model(u.data_ptr(), np.zeros(5), np.ones(5), np.ones(6))
        with pytest.raises(fk.FFTKError) as e:
            fk.tarang_ns_step(plan, u.data_ptr(), fk.make_params(1e-3, 1e-3, sgs_model=model), 1, False, stream())
        assert e.value.status == fk.FFTK_ERR_UNSUPPORTED_SIZE
    finally:
        fk.fftk_plan_destroy(plan)
    plan = fk.fftk_plan_create(1536, 1536, 1536)
    try:
        with pytest.raises(fk.FFTKError) as e:
            fk.tarang_ns_step(plan, u.data_ptr(), fk.make_params(1e-3, 1e-3), 1, False, stream())
        assert e.value.status == fk.FFTK_ERR_UNSUPPORTED_SIZE
    finally:
        fk.fftk_plan_destroy(plan)
    for bad in ((5, 8, 8), (6, 6, 6), (8, 8, 9), (6144, 2, 12)):
        with pytest.raises(fk.FFTKError):
            fk.fftk_plan_create(*bad)
