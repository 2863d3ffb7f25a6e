"""Pins for the oracle's transforms (Sec. 2.1 Eq. (1); Sec. 3 pass order).

Each test compares the FFT-based oracle with something it does not share code
with: brute-force sums, closed forms, numpy's FFT, or invariants.
"""
import itertools

import numpy as np
import pytest

import synth

RNG = np.random.default_rng(12345)


def _crand(shape):
    return RNG.standard_normal(shape) + 1j * RNG.standard_normal(shape)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64, 128])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft1d_equals_direct_dft(oracle_mod, n, sign):
    x = _crand(n)
    a = oracle_mod.fft1d(x, sign)
    b = oracle_mod.dft1d(x, sign)
    assert np.max(np.abs(a - b)) <= 1e-13 * max(1.0, np.max(np.abs(b)))


@pytest.mark.parametrize("n", [3, 5, 12, 16])
def test_dft1d_closed_forms(oracle_mod, n):
    # delta at j0 -> exp(-2 pi i j0 k / n); exp(+2 pi i k0 j / n) -> n delta(k - k0)
    j0, k0 = 1, n - 1
    d = np.zeros(n, complex)
    d[j0] = 1
    k = np.arange(n)
    assert np.allclose(oracle_mod.dft1d(d, -1), np.exp(-2j * np.pi * j0 * k / n), atol=1e-14)
    e = np.exp(2j * np.pi * k0 * k / n)
    want = np.zeros(n, complex)
    want[k0] = n
    assert np.allclose(oracle_mod.dft1d(e, -1), want, atol=1e-12)


def test_fft1d_rejects_non_power_of_two(oracle_mod):
    with pytest.raises(RuntimeError):
        oracle_mod.fft1d(np.zeros(12, complex))


def _direct_rfft3(f):
    """Brute force: the forward DFT as three explicit DFT-matrix products."""
    nx, ny, nz = f.shape
    Wx = np.exp(-2j * np.pi * np.outer(np.arange(nx), np.arange(nx)) / nx)
    Wy = np.exp(-2j * np.pi * np.outer(np.arange(ny), np.arange(ny)) / ny)
    Wz = np.exp(-2j * np.pi * np.outer(np.arange(nz // 2 + 1), np.arange(nz)) / nz)
    F = np.einsum("ai,bj,cl,ijl->abc", Wx, Wy, Wz, f.astype(complex))
    return F / (nx * ny * nz)


SMALL = [1, 2, 4, 8, 16]


@pytest.mark.parametrize("shape", [s for s in itertools.product(SMALL, SMALL, SMALL) if s[2] >= 2][::3])
def test_rfft3_equals_brute_force(oracle_mod, shape):
    f = RNG.standard_normal(shape)
    F = oracle_mod.rfft3(f)
    G = _direct_rfft3(f)
    assert F.shape == G.shape
    assert np.max(np.abs(F - G)) <= 1e-14 * max(1.0, np.max(np.abs(G))) * 10


@pytest.mark.parametrize("shape", [(32, 32, 32), (64, 64, 64), (8, 32, 16), (128, 4, 64), (2, 2, 128)])
def test_rfft3_matches_numpy(oracle_mod, shape):
    f = RNG.standard_normal(shape)
    F = oracle_mod.rfft3(f)
    G = np.fft.rfftn(f) / f.size
    assert np.max(np.abs(F - G)) <= 1e-15 * np.sqrt(np.log2(f.size)) * 10
    back = oracle_mod.irfft3(F, shape[2])
    assert np.max(np.abs(back - np.fft.irfftn(G * f.size, s=shape, axes=(0, 1, 2)))) <= 1e-12


@pytest.mark.parametrize("k0", [(2, 3, 5), (0, 7, 0), (3, -4, 1), (-8, 0, 8)])
def test_single_mode_cos_closed_form(oracle_mod, k0):
    # f = cos(k0 . x): stored coefficients are exactly 1/2 at +k0 (and -k0 when
    # k_z = 0 or N/2, where both are stored), zero elsewhere.
    n = 16
    a, b, c = k0
    g = 2 * np.pi * np.arange(n) / n
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    f = np.cos(a * X + b * Y + c * Z)
    F = oracle_mod.rfft3(f)
    want = np.zeros_like(F)
    want[a % n, b % n, c] += 0.5
    if c == 0 or c == n // 2:
        want[(-a) % n, (-b) % n, c] += 0.5
    assert np.max(np.abs(F - want)) < 1e-14


def test_single_mode_sin_sign(oracle_mod):
    # sin(k.x) = (e^{ik.x} - e^{-ik.x}) / (2i): coefficient at +k is -i/2
    n = 8
    g = 2 * np.pi * np.arange(n) / n
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    F = oracle_mod.rfft3(np.sin(X + 2 * Y + 3 * Z))
    assert abs(F[1, 2, 3] - (-0.5j)) < 1e-15
    F[1, 2, 3] = 0
    assert np.max(np.abs(F)) < 1e-15


def test_parseval_and_hermitian_plane(oracle_mod):
    n = (16, 8, 32)
    f = RNG.standard_normal(n)
    F = oracle_mod.rfft3(f)
    w = np.full(F.shape[-1], 2.0)
    w[0] = 1.0
    w[-1] = 1.0
    lhs = np.mean(f**2)
    rhs = np.sum(w * np.abs(F) ** 2)
    assert abs(lhs - rhs) <= 1e-13 * lhs
    # k_z = 0 plane: F(-kx, -ky, 0) = conj F(kx, ky, 0)
    P = F[:, :, 0]
    Pm = np.conj(P[(-np.arange(n[0])) % n[0]][:, (-np.arange(n[1])) % n[1]])
    assert np.max(np.abs(P - Pm)) < 1e-15


def test_round_trip_and_linearity(oracle_mod):
    shape = (16, 32, 8)
    f = RNG.standard_normal(shape)
    g = RNG.standard_normal(shape)
    F, G = oracle_mod.rfft3(f), oracle_mod.rfft3(g)
    assert np.max(np.abs(oracle_mod.irfft3(F, shape[2]) - f)) < 1e-13
    H = oracle_mod.rfft3(2.5 * f - 0.75 * g)
    assert np.max(np.abs(H - (2.5 * F - 0.75 * G))) < 1e-14


def test_shift_theorem(oracle_mod):
    # f(x - x0) with x0 = 2 pi s/N has coefficients F(k) exp(-i k . x0)
    shape = (8, 16, 16)
    s = (3, 5, 7)
    f = RNG.standard_normal(shape)
    fs = np.roll(f, s, axis=(0, 1, 2))
    F, Fs = oracle_mod.rfft3(f), oracle_mod.rfft3(fs)
    a = np.arange(shape[0])[:, None, None]
    b = np.arange(shape[1])[None, :, None]
    c = np.arange(shape[2] // 2 + 1)[None, None, :]
    ph = np.exp(-2j * np.pi * (a * s[0] / shape[0] + b * s[1] / shape[1] + c * s[2] / shape[2]))
    assert np.max(np.abs(Fs - F * ph)) < 1e-14


def test_irfft3_drops_imaginary_dc_and_nyquist_of_lines(oracle_mod):
    # Line-wise c2r keeps only Re of the k_z = 0 and k_z = N/2 coefficients of
    # each z line: an imaginary constant contributes nothing.
    n = 8
    F = np.zeros((n, n, n // 2 + 1), complex)
    F[0, 0, 0] = 2.0 + 5.0j
    F[0, 0, n // 2] = 1.0 - 3.0j
    out = oracle_mod.irfft3(F, n)
    l = np.arange(n)
    want = 2.0 + 1.0 * (-1.0) ** l
    assert np.max(np.abs(out - want[None, None, :])) < 1e-14


def test_direct_coefficient_and_point_sums(oracle_mod):
    shape = (8, 4, 16)
    f = synth.uniform_pm1(0, 0, shape)
    F = oracle_mod.rfft3(f.astype(np.float64))
    for (a, b, c) in [(0, 0, 0), (1, 3, 8), (7, 2, 5), (4, 0, 1)]:
        assert abs(oracle_mod.rfft3_coeff(f, a, b, c) - F[a, b, c]) < 1e-15
    F32 = F.astype(np.complex64)
    back = oracle_mod.irfft3(F32.astype(np.complex128), shape[2])
    for (i, j, l) in [(0, 0, 0), (7, 3, 15), (2, 1, 9)]:
        assert abs(oracle_mod.irfft3_point(F32, shape[2], i, j, l) - back[i, j, l]) < 1e-12


def test_rejects_bad_shapes(oracle_mod):
    with pytest.raises(RuntimeError):
        oracle_mod.rfft3(np.zeros((5, 8, 8)))
    with pytest.raises(RuntimeError):
        oracle_mod.rfft3(np.zeros((8, 9, 8)))
    with pytest.raises(RuntimeError):
        oracle_mod.rfft3(np.zeros((8, 8, 1)))


@pytest.mark.parametrize("shape", [(6, 12, 24), (3, 8, 6), (12, 6, 48), (24, 3, 12)])
def test_radix3_lengths_match_numpy_and_brute_force(oracle_mod, shape):
    # dimensions 3 * 2^m (the paper's 768, 1536, 3072 grids): numpy's FFT and
    # the three explicit DFT matrices
    f = synth.uniform_pm1(9, 0, shape).astype(np.float64)
    F = oracle_mod.rfft3(f)
    assert np.max(np.abs(F - np.fft.rfftn(f) / f.size)) < 1e-15
    assert np.max(np.abs(F - _direct_rfft3(f))) < 1e-15
    assert np.max(np.abs(oracle_mod.irfft3(F, shape[2]) - f)) < 1e-14
    for (a, b, c) in [(0, 0, 0), (1, 2, 3), (shape[0] - 1, shape[1] - 1, shape[2] // 2)]:
        assert abs(oracle_mod.rfft3_coeff(f.astype(np.float32), a, b, c) - F[a, b, c]) < 1e-14
