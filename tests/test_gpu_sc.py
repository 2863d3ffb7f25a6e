"""GPU parity of the mixed-basis transforms (fftk_forward / fftk_inverse:
Fourier, sine and cosine axes; paper Sec. 2.1) against the FP64 oracle,
through the C ABI.

Tolerance: a sine/cosine pass is one FP32 FFT of the line's length plus a
pre-permutation and a post-twiddle (two rounded products), so the transform
keeps the Fourier bar: relative L2 <= 2e-6 and 1e-5 of the largest
coefficient per element.
"""
import numpy as np
import pytest

import synth
from gpu_helpers import from_dev_c64, rel_l2, stream, sync

pytestmark = pytest.mark.gpu

BASES = ["SFF", "CFF", "SSF", "CSF", "SCF", "CCF", "SSS", "CCS", "SCC", "CCC", "SSC", "FFF"]


@pytest.fixture(scope="module")
def fk():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_07801_gb300 import build as b

    b.build()
    import paper_1805_07801_gb300 as m

    return m


def _spec_shape(shape, basis):
    nx, ny, nz = shape
    return (nx, ny, nz // 2 + 1) if basis[2] == "F" else (nx, ny, nz)


def _gpu_forward(fk, plan, f32, basis, batch=1):
    import torch

    dev = torch.device("cuda:0")
    x = torch.from_numpy(np.ascontiguousarray(f32)).to(dev)
    spec = _spec_shape(f32.shape[-3:], basis)
    if basis[2] == "F":
        out = torch.empty((batch,) + spec + (2,), dtype=torch.float32, device=dev)
    else:
        out = torch.empty((batch,) + spec, dtype=torch.float32, device=dev)
    fk.fftk_forward(plan, basis, x.data_ptr(), out.data_ptr(), batch, stream())
    sync()
    if basis[2] == "F":
        return from_dev_c64(out), out
    return out.cpu().numpy().astype(np.float64), out


def _gpu_inverse(fk, plan, spec_dev, shape, basis, batch=1):
    import torch

    y = torch.empty((batch,) + tuple(shape), dtype=torch.float32, device="cuda:0")
    before = spec_dev.clone()
    fk.fftk_inverse(plan, basis, spec_dev.data_ptr(), y.data_ptr(), batch, stream())
    sync()
    assert torch.equal(before, spec_dev)  # the input is not modified
    return y.cpu().numpy()


@pytest.mark.parametrize("basis", BASES)
@pytest.mark.parametrize("shape", [(8, 16, 32), (32, 32, 32), (64, 8, 128), (2, 4, 2)])
def test_forward_and_inverse_match_oracle(fk, oracle_mod, basis, shape):
    f = synth.uniform_pm1(11, 0, shape)
    plan = fk.fftk_plan_create(*shape)
    try:
        got, dev_spec = _gpu_forward(fk, plan, f[None], basis)
        want = oracle_mod.transform3(f.astype(np.float64), basis)
        assert rel_l2(got[0], want) < 2e-6
        assert np.max(np.abs(got[0] - want)) < 1e-5 * np.max(np.abs(want))
        back = _gpu_inverse(fk, plan, dev_spec, shape, basis)
        assert rel_l2(back[0], f) < 2e-6
        # inverse of the oracle's spectrum against the oracle's inverse
        import torch

        if basis[2] == "F":
            w = np.ascontiguousarray(want.astype(np.complex64))
            sd = torch.from_numpy(w.view(np.float32).reshape(w.shape + (2,))).to("cuda:0")[None]
        else:
            sd = torch.from_numpy(np.ascontiguousarray(want.real, dtype=np.float32)).to("cuda:0")[None]
        inv = _gpu_inverse(fk, plan, sd, shape, basis)
        assert rel_l2(inv[0], oracle_mod.itransform3(want, shape[2], basis)) < 2e-6
    finally:
        fk.fftk_plan_destroy(plan)


def test_fff_equals_r2c_bitwise(fk):
    import torch

    shape = (16, 32, 64)
    f = synth.uniform_pm1(12, 0, shape)
    plan = fk.fftk_plan_create(*shape)
    try:
        x = torch.from_numpy(f).to("cuda:0")
        a = torch.empty(shape[:2] + (shape[2] // 2 + 1, 2), device="cuda:0")
        b = torch.empty_like(a)
        fk.fftk_forward(plan, "FFF", x.data_ptr(), a.data_ptr(), 1, stream())
        fk.fftk_r2c(plan, x.data_ptr(), b.data_ptr(), 1, stream())
        sync()
        assert torch.equal(a, b)
    finally:
        fk.fftk_plan_destroy(plan)


def test_batched_and_long_axes(fk, oracle_mod):
    # a batch of two, and the longest sine/cosine lines (4096 points)
    shape = (16, 8, 32)
    f = np.stack([synth.uniform_pm1(13, i, shape) for i in range(2)])
    plan = fk.fftk_plan_create(*shape)
    try:
        got, _ = _gpu_forward(fk, plan, f, "SSF", batch=2)
    finally:
        fk.fftk_plan_destroy(plan)
    for i in range(2):
        assert rel_l2(got[i], oracle_mod.transform3(f[i].astype(np.float64), "SSF")) < 2e-6
    for shape, basis in (((4096, 2, 2), "SFF"), ((2, 2, 4096), "SSS"), ((2, 4096, 2), "CCF")):
        g = synth.uniform_pm1(14, 0, shape)
        plan = fk.fftk_plan_create(*shape)
        try:
            got, dev_spec = _gpu_forward(fk, plan, g[None], basis)
            back = _gpu_inverse(fk, plan, dev_spec, shape, basis)
        finally:
            fk.fftk_plan_destroy(plan)
        want = oracle_mod.transform3(g.astype(np.float64), basis)
        assert rel_l2(got[0], want) < 2e-6, (shape, basis)
        assert rel_l2(back[0], g) < 2e-6


@pytest.mark.parametrize("basis", ["SFF", "CCS"])
def test_full_size_sampled_coefficients(fk, oracle_mod, basis):
    # 512^3: coefficients at sampled (a, b, c) against the oracle's definition,
    # plus the round trip
    import torch

    n = 512
    dev = torch.device("cuda:0")
    plan = fk.fftk_plan_create(n, n, n)
    try:
        x = torch.empty((n, n, n), dtype=torch.float32, device=dev)
        fk.fftk_fill_uniform(x.data_ptr(), x.numel(), 21, 0, stream())
        spec = _spec_shape((n, n, n), basis)
        if basis[2] == "F":
            out = torch.empty(spec + (2,), dtype=torch.float32, device=dev)
        else:
            out = torch.empty(spec, dtype=torch.float32, device=dev)
        fk.fftk_forward(plan, basis, x.data_ptr(), out.data_ptr(), 1, stream())
        y = torch.empty_like(x)
        fk.fftk_inverse(plan, basis, out.data_ptr(), y.data_ptr(), 1, stream())
        sync()
        xh = x.cpu().numpy()
        oh = out.cpu().numpy()
        err = float(torch.linalg.vector_norm((y - x).double()) / torch.linalg.vector_norm(x.double()))
    finally:
        fk.fftk_plan_destroy(plan)
    assert err < 2e-6
    rng = np.random.default_rng(0)
    picks = [(0, 0, 0), (n - 1, n - 1, spec[2] - 1), (1, 2, 3)]
    picks += [tuple(int(rng.integers(0, d)) for d in spec) for _ in range(5)]
    scale = 1.0 / np.sqrt(3.0 * n**3)  # rms of a coefficient of uniform(-1, 1) input, about
    for a, b, c in picks:
        want = oracle_mod.transform3_coeff(xh, basis, a, b, c)
        got = complex(oh[a, b, c, 0], oh[a, b, c, 1]) if basis[2] == "F" else complex(oh[a, b, c], 0.0)
        assert abs(got - want) < 1e-4 * scale, (a, b, c, got, want)


def test_argument_errors(fk):
    import torch

    plan = fk.fftk_plan_create(8, 1, 8)
    try:
        x = torch.zeros((8, 1, 8), device="cuda:0")
        o = torch.zeros((8, 1, 8, 2), device="cuda:0")
        for bad in ("FSF", "FFS", "SFS", "SSF", [0, 0, 7]):  # SSF: a sine axis of one point
            with pytest.raises(fk.FFTKError):
                fk.fftk_forward(plan, bad, x.data_ptr(), o.data_ptr(), 1, stream())
        with pytest.raises(fk.FFTKError):  # in place
            fk.fftk_forward(plan, "SFF", x.data_ptr(), x.data_ptr(), 1, stream())
    finally:
        fk.fftk_plan_destroy(plan)
