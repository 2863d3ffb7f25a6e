"""GPU input generators and the random-phase initial field, through the C ABI.

The GPU SplitMix64 must reproduce the numpy generator in synth/ exactly for
the uniform fields (integer arithmetic), and the FP64 Box-Muller normals up to
the last bit of FP32 where the device and host libm differ by an ulp in FP64.
The initial field is then compared with the oracle's, built from the numpy
normals, within the FP32 rounding of the transform chain.
"""
import numpy as np
import pytest

import synth
from gpu_helpers import empty_c64, empty_real, from_dev_c64, rel_l2, stream, sync

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


def test_uniform_bit_exact(fk):
    shape = (37, 64, 64)
    for seed, field in [(0, 0), (5, 3)]:
        t = empty_real(shape)
        fk.fftk_fill_uniform(t.data_ptr(), t.numel(), seed, field, stream())
        sync()
        assert np.array_equal(t.cpu().numpy(), synth.uniform_pm1(seed, field, shape))


def test_normal_matches_numpy_generator(fk):
    shape = (64, 64, 64)
    t = empty_real(shape)
    fk.fftk_fill_normal(t.data_ptr(), t.numel(), 0, 1, stream())
    sync()
    g = t.cpu().numpy()
    h = synth.normal(0, 1, shape).astype(np.float32)
    diff = g != h
    assert diff.mean() < 1e-4
    if diff.any():
        assert np.max(np.abs(g[diff] - h[diff]) / np.abs(h[diff])) < 2.0**-22


def test_fill_rejects_bad_arguments(fk):
    t = empty_real((16,))
    for args in [(t.data_ptr(), 16, -1, 0), (t.data_ptr(), 16, 0, 16), (0, 16, 0, 0), (t.data_ptr() + 2, 4, 0, 0)]:
        with pytest.raises(fk.FFTKError) as e:
            fk.fftk_fill_normal(*args, stream())
        assert e.value.status == fk.FFTK_ERR_INVALID_ARG


@pytest.mark.parametrize("n,k0", [(32, 2.0), (64, 4.0)])
def test_ic_random_matches_oracle(fk, oracle_mod, n, k0):
    normals = empty_real((3, n, n, n))
    for f in range(3):
        fk.fftk_fill_normal(normals[f].data_ptr(), n**3, 0, f, stream())
    u = empty_c64((3, n, n, n // 2 + 1))
    plan = fk.fftk_plan_create(n, n, n)
    try:
        fk.tarang_ic_random(plan, normals.data_ptr(), u.data_ptr(), k0, 0.5, stream())
        E, _, EK = fk.tarang_diag(plan, u.data_ptr(), 0.0, stream())
    finally:
        fk.fftk_plan_destroy(plan)
    ug = from_dev_c64(u)
    uo = oracle_mod.ic_random(synth.normal_fields(0, 3, (n, n, n)), k0=k0, E0=0.5)
    assert rel_l2(ug, uo) < 1e-5
    assert abs(E - 0.5) < 1e-6
    # exactly Hermitian on k_z = 0
    P = ug[:, :, :, 0]
    Pm = np.conj(P[:, (-np.arange(n)) % n][:, :, (-np.arange(n)) % n])
    assert np.array_equal(P, Pm)
