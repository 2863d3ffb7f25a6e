"""GPU parity of the 3D R2C / C2R transforms (fftk_r2c, fftk_c2r) against the
FP64 oracle, through the C ABI.

Tolerance: FP32 arithmetic with correctly rounded FP32 twiddles; the error of
a Cooley-Tukey transform grows at most with the number of radix-2 levels,
relative L2 <= ~u log2(N^3) (u = 2^-24): 1.8e-6 at 1024^3.  Every case uses
the bound 2e-6 on relative L2 and 1e-5 * max|F| per element.
"""
import numpy as np
import pytest

import synth
from gpu_helpers import empty_c64, empty_real, from_dev_c64, rel_l2, stream, sync, to_dev_c64, to_dev_real

pytestmark = pytest.mark.gpu

REL = 2e-6


@pytest.fixture(scope="module")
def fk():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_07801_gb300 import build as b

    b.build()
    import paper_1805_07801_gb300 as m

    return m


class Plan:
    def __init__(self, fk, shape):
        self.fk = fk
        self.h = fk.fftk_plan_create(*shape)

    def __enter__(self):
        return self.h

    def __exit__(self, *a):
        self.fk.fftk_plan_destroy(self.h)


def _spec_shape(shape, batch=None):
    s = (shape[0], shape[1], shape[2] // 2 + 1)
    return s if batch is None else (batch,) + s


def gpu_r2c(fk, plan, f, batch=None):
    x = to_dev_real(f)
    F = empty_c64(_spec_shape(f.shape[-3:], batch))
    fk.fftk_r2c(plan, x.data_ptr(), F.data_ptr(), batch or 1, stream())
    sync()
    return from_dev_c64(F)


def gpu_c2r(fk, plan, F, nz, batch=None):
    Fd = to_dev_c64(F)
    out = empty_real(F.shape[:-1] + (nz,))
    fk.fftk_c2r(plan, Fd.data_ptr(), out.data_ptr(), batch or 1, stream())
    sync()
    return out.cpu().numpy()


SHAPES = [
    (1, 1, 2), (2, 2, 2), (1, 1, 8), (8, 4, 2), (4, 8, 16), (16, 1, 32), (64, 64, 64),
    (32, 128, 16), (128, 16, 256), (2, 512, 4), (1024, 2, 2), (8, 8, 4096), (4, 2048, 4),
    (2048, 2, 4), (4096, 1, 2), (1, 4096, 2), (256, 256, 8),
    # 512-point x lines with an even row stride ny (nz/2+1) take the TMA
    # pass (ragged last tile at 40 columns); the others are ragged tiles of
    # the plain pass for 1024- and 2048-point lines
    (1024, 2, 8), (512, 8, 8), (2048, 1, 8), (4, 1024, 8),
    # row lengths Q with a remainder past the last full tile (y passes with
    # Q = nz/2 + 1 = 129, 33, 17 and 25 columns; an x pass with Q = 30)
    (8, 256, 256), (4, 512, 64), (2, 1024, 32), (16, 256, 48), (256, 6, 8),
]


@pytest.mark.parametrize("shape", SHAPES)
def test_r2c_matches_oracle(fk, oracle_mod, shape):
    f = synth.uniform_pm1(0, 0, shape)
    with Plan(fk, shape) as plan:
        Fg = gpu_r2c(fk, plan, f)
    Fo = oracle_mod.rfft3(f.astype(np.float64))
    assert rel_l2(Fg, Fo) < REL
    assert np.max(np.abs(Fg - Fo)) <= 1e-5 * np.max(np.abs(Fo))


@pytest.mark.parametrize("shape", SHAPES)
def test_c2r_matches_oracle(fk, oracle_mod, shape):
    f = synth.uniform_pm1(1, 0, shape)
    F = oracle_mod.rfft3(f.astype(np.float64)).astype(np.complex64)
    with Plan(fk, shape) as plan:
        g = gpu_c2r(fk, plan, F, shape[2])
    go = oracle_mod.irfft3(F.astype(np.complex128), shape[2])
    assert rel_l2(g, go) < REL
    assert np.max(np.abs(g - go)) <= 1e-5 * np.max(np.abs(go))


@pytest.mark.parametrize("shape", [(8, 16, 8), (32, 4, 64), (1, 1, 16)])
def test_c2r_non_hermitian_input_is_line_wise(fk, oracle_mod, shape):
    # arbitrary complex input: both sides take the real part line by line
    # after the x and y passes (Im of each z line's k_z = 0, nz/2 dropped)
    rng = np.random.default_rng(11)
    hs = _spec_shape(shape)
    F = (rng.standard_normal(hs) + 1j * rng.standard_normal(hs)).astype(np.complex64)
    with Plan(fk, shape) as plan:
        g = gpu_c2r(fk, plan, F, shape[2])
    go = oracle_mod.irfft3(F.astype(np.complex128), shape[2])
    assert rel_l2(g, go) < REL


@pytest.mark.parametrize("shape, B", [((16, 32, 8), 3), ((512, 4, 4), 2), ((1024, 4, 4), 2), ((8, 512, 4), 2)])
def test_batched_equals_separate(fk, oracle_mod, shape, B):
    f = np.stack([synth.uniform_pm1(0, b, shape) for b in range(B)])
    with Plan(fk, shape) as plan:
        Fg = gpu_r2c(fk, plan, f, batch=B)
        back = gpu_c2r(fk, plan, Fg, shape[2], batch=B)
        for b in range(B):
            assert np.array_equal(Fg[b], gpu_r2c(fk, plan, f[b]))
    Fo = oracle_mod.rfft3(f.astype(np.float64))
    assert rel_l2(Fg, Fo) < REL
    assert rel_l2(back, f * np.float32(1.0)) < REL


def test_inputs_preserved_and_deterministic(fk):
    import torch

    shape = (64, 32, 128)
    f = synth.uniform_pm1(2, 0, shape)
    with Plan(fk, shape) as plan:
        x = to_dev_real(f)
        x0 = x.clone()
        F1 = empty_c64(_spec_shape(shape))
        F2 = empty_c64(_spec_shape(shape))
        fk.fftk_r2c(plan, x.data_ptr(), F1.data_ptr(), 1, stream())
        fk.fftk_r2c(plan, x.data_ptr(), F2.data_ptr(), 1, stream())
        Fc = F1.clone()
        o1 = empty_real(shape)
        o2 = empty_real(shape)
        fk.fftk_c2r(plan, F1.data_ptr(), o1.data_ptr(), 1, stream())
        fk.fftk_c2r(plan, F1.data_ptr(), o2.data_ptr(), 1, stream())
        sync()
        assert torch.equal(x, x0)
        assert torch.equal(F1, F2)
        assert torch.equal(F1, Fc)
        assert torch.equal(o1, o2)


def test_argument_errors_on_device(fk):
    import torch

    shape = (16, 16, 16)
    with Plan(fk, shape) as plan:
        buf = torch.zeros(4 * 16 * 16 * 16 * 4, dtype=torch.float32, device="cuda:0")
        p = buf.data_ptr()
        with pytest.raises(fk.FFTKError) as e:
            fk.fftk_r2c(plan, p, p + 64, 1, stream())  # overlapping
        assert e.value.status == fk.FFTK_ERR_INVALID_ARG
        with pytest.raises(fk.FFTKError) as e:
            fk.fftk_r2c(plan, p + 4, p + 4 * 16**3 * 4, 1, stream())  # misaligned
        assert e.value.status == fk.FFTK_ERR_INVALID_ARG
        with pytest.raises(fk.FFTKError) as e:
            fk.fftk_c2r(plan, p, p, 1, stream())
        assert e.value.status == fk.FFTK_ERR_INVALID_ARG
        with pytest.raises(fk.FFTKError) as e:
            fk.fftk_r2c(plan, p, p + 4 * 16**3 * 4, 0, stream())
        assert e.value.status == fk.FFTK_ERR_INVALID_ARG


def test_caller_workspace_and_launch_count(fk, oracle_mod):
    import torch

    shape = (32, 16, 64)
    f = synth.uniform_pm1(3, 0, shape)
    with Plan(fk, shape) as plan:
        nb = fk.fftk_workspace_bytes(plan, 1)
        assert nb == 2 * 32 * 16 * 33 * 8  # two spectra: both strided passes run out of place
        ws = torch.empty(nb // 4, dtype=torch.float32, device="cuda:0")
        fk.fftk_set_workspace(plan, ws.data_ptr(), nb)
        n0 = fk.fftk_launch_count(plan)
        F = gpu_r2c(fk, plan, f)
        assert fk.fftk_launch_count(plan) - n0 == 3
        g = gpu_c2r(fk, plan, F, shape[2])
        assert fk.fftk_launch_count(plan) - n0 == 6
        assert rel_l2(g, f) < REL
        small = torch.empty(16, dtype=torch.float32, device="cuda:0")
        fk.fftk_set_workspace(plan, small.data_ptr(), 64)
        with pytest.raises(fk.FFTKError) as e:
            gpu_c2r(fk, plan, F, shape[2])
        assert e.value.status == fk.FFTK_ERR_INVALID_ARG


def test_smaller_caller_workspaces_run_the_passes_in_place(fk, oracle_mod):
    # one spectrum of workspace: c2r runs its y pass in place; less than one:
    # r2c runs both strided passes in place in its output (c2r then fails)
    import torch

    shape = (32, 16, 64)
    f = synth.uniform_pm1(4, 0, shape)
    Fo = oracle_mod.rfft3(f.astype(np.float64))
    with Plan(fk, shape) as plan:
        one = fk.fftk_workspace_bytes(plan, 1) // 2
        ws = torch.empty(one // 4, dtype=torch.float32, device="cuda:0")
        fk.fftk_set_workspace(plan, ws.data_ptr(), one)
        Fg = gpu_r2c(fk, plan, f)
        g = gpu_c2r(fk, plan, Fg.astype(np.complex64), shape[2])
        assert rel_l2(Fg, Fo) < REL and rel_l2(g, f) < REL
        small = torch.empty(16, dtype=torch.float32, device="cuda:0")
        fk.fftk_set_workspace(plan, small.data_ptr(), 64)
        assert rel_l2(gpu_r2c(fk, plan, f), Fo) < REL
        with pytest.raises(fk.FFTKError) as e:
            gpu_c2r(fk, plan, Fg.astype(np.complex64), shape[2])
        assert e.value.status == fk.FFTK_ERR_INVALID_ARG


def test_profile_records_each_pass(fk):
    shape = (64, 64, 64)
    f = synth.uniform_pm1(0, 0, shape)
    with Plan(fk, shape) as plan:
        fk.fftk_profile_enable(plan, True)
        gpu_r2c(fk, plan, f)
        for name in ["z_r2c", "y_fwd", "x_fwd"]:
            ms, n = fk.fftk_profile_read(plan, fk.kernel_index(name))
            assert n == 1 and ms > 0.0
        fk.fftk_profile_enable(plan, False)


def test_full_size_1024_pair(fk, oracle_mod):
    """The 1024^3 FP32 pair in the benchmark's launch configuration: round
    trip, Parseval, and sampled coefficients / points by direct O(N^3) sums."""
    import torch

    n = 1024
    shape = (n, n, n)
    f = synth.uniform_pm1(0, 0, shape)
    with Plan(fk, shape) as plan:
        x = to_dev_real(f)
        F = empty_c64(_spec_shape(shape))
        back = empty_real(shape)
        fk.fftk_r2c(plan, x.data_ptr(), F.data_ptr(), 1, stream())
        fk.fftk_c2r(plan, F.data_ptr(), back.data_ptr(), 1, stream())
        sync()
        rt = (torch.linalg.vector_norm((back - x).double()) / torch.linalg.vector_norm(x.double())).item()
        assert rt < REL
        Fd = F.double()
        w = torch.full((n // 2 + 1,), 2.0, dtype=torch.float64, device=F.device)
        w[0] = 1.0
        w[-1] = 1.0
        spec = ((Fd[..., 0] ** 2 + Fd[..., 1] ** 2) * w).sum().item()
        phys = (x.double() ** 2).mean().item()
        assert abs(spec - phys) < 1e-6 * phys
        pts = [(0, 0, 0), (5, 1000, 77), (1023, 1, 1023)]
        back_pts = [back[i, j, l].item() for (i, j, l) in pts]
        del back, Fd
        Fh = from_dev_c64(F)
    rms = float(np.sqrt(np.mean(np.abs(Fh) ** 2)))
    for (a, b, c) in [(0, 0, 0), (1, 2, 3), (1023, 512, 511), (300, 700, 512)]:
        want = oracle_mod.rfft3_coeff(f, a, b, c)
        assert abs(Fh[a, b, c] - want) < 1e-5 * rms
    for (i, j, l), got in zip(pts, back_pts):
        # the oracle's direct inverse sum of the GPU spectrum: recovers the input
        # (checks r2c) and equals the GPU c2r output (checks c2r)
        want = oracle_mod.irfft3_point(Fh, n, i, j, l)
        assert abs(want - f[i, j, l]) < 1e-5
        assert abs(got - want) < 1e-5
