"""Pins for the oracle's sine and cosine bases (Sec. 2.1, Eq. (2b, 2c)) and
the mixed-basis 3D transforms FFF, SFF, SSF, SSS.

A line of n points s_j = (j + 1/2) pi / n on [0, pi]; inverse
f(s_j) = sum_k fhat_k 2 sin(k s_j) (k = 1..n) or 2 cos(k s_j) (k = 0..n-1).
Checked against scipy's DCT-II/DST-II (a library routine for the special
case of one line), single-mode closed forms, round trips, the Fourier-only
case against the oracle's own FFF transform and numpy, and separability.
"""
import numpy as np
import pytest

import synth


def _s(n):
    return (np.arange(n) + 0.5) * np.pi / n


@pytest.mark.parametrize("n", [1, 2, 3, 8, 12, 64])
def test_cosine_forward_matches_scipy_dct2(oracle_mod, n):
    sfft = pytest.importorskip("scipy.fft")
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    got = oracle_mod.sc1d(x, "C", -1)
    y = sfft.dct(x.real, type=2) + 1j * sfft.dct(x.imag, type=2)  # 2 sum x cos(pi k (2j+1) / 2n)
    want = y / (2 * n)
    want[0] *= 0.5
    assert np.max(np.abs(got - want)) < 1e-14 * max(1.0, np.max(np.abs(want)))


@pytest.mark.parametrize("n", [1, 2, 3, 8, 12, 64])
def test_sine_forward_matches_scipy_dst2(oracle_mod, n):
    sfft = pytest.importorskip("scipy.fft")
    rng = np.random.default_rng(100 + n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    got = oracle_mod.sc1d(x, "S", -1)
    y = sfft.dst(x.real, type=2) + 1j * sfft.dst(x.imag, type=2)  # 2 sum x sin(pi (k+1)(2j+1) / 2n)
    want = y / (2 * n)
    want[-1] *= 0.5
    assert np.max(np.abs(got - want)) < 1e-14 * max(1.0, np.max(np.abs(want)))


@pytest.mark.parametrize("n", [8, 16, 10])
def test_single_modes(oracle_mod, n):
    s = _s(n)
    c = oracle_mod.sc1d(2 * np.cos(3 * s), "C", -1)
    assert np.max(np.abs(c - np.eye(n)[3])) < 1e-14
    c0 = oracle_mod.sc1d(2 * np.ones(n), "C", -1)  # the k = 0 mode: 2 cos(0) = 2
    assert np.max(np.abs(c0 - np.eye(n)[0])) < 1e-14
    sn = oracle_mod.sc1d(2 * np.sin(5 * s), "S", -1)
    assert np.max(np.abs(sn - np.eye(n)[4])) < 1e-14
    top = oracle_mod.sc1d(2 * np.sin(n * s), "S", -1)  # 2 sin(n s_j) = 2 (-1)^j
    assert np.max(np.abs(top - np.eye(n)[n - 1])) < 1e-14
    # and the inverse synthesises them back
    assert np.max(np.abs(oracle_mod.sc1d(np.eye(n)[3], "C", +1) - 2 * np.cos(3 * s))) < 1e-14
    assert np.max(np.abs(oracle_mod.sc1d(np.eye(n)[n - 1], "S", +1) - 2 * np.sin(n * s))) < 1e-14


@pytest.mark.parametrize("kind", ["S", "C"])
@pytest.mark.parametrize("n", [1, 2, 7, 16, 128])
def test_round_trip(oracle_mod, kind, n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    back = oracle_mod.sc1d(oracle_mod.sc1d(x, kind, -1), kind, +1)
    assert np.max(np.abs(back - x)) < 1e-13


def test_fff_is_the_fourier_transform(oracle_mod):
    f = synth.uniform_pm1(3, 0, (8, 16, 32)).astype(np.float64)
    got = oracle_mod.transform3(f, "FFF")
    assert np.max(np.abs(got - np.fft.rfftn(f) / f.size)) < 1e-15
    assert np.max(np.abs(got - oracle_mod.rfft3(f))) < 1e-15
    assert np.max(np.abs(oracle_mod.itransform3(got, 32, "FFF") - f)) < 1e-14


@pytest.mark.parametrize("basis", ["SFF", "CFF", "SSF", "CSF", "SSS", "CCS", "SCC"])
def test_mixed_bases_are_separable(oracle_mod, basis):
    sfft = pytest.importorskip("scipy.fft")
    nx, ny, nz = 8, 16, 8
    f = synth.uniform_pm1(4, 0, (nx, ny, nz)).astype(np.float64)

    def sc_axis(a, axis, kind):  # scipy DCT-II / DST-II along an axis, in the basis' normalisation
        n = a.shape[axis]
        t = sfft.dst if kind == "S" else sfft.dct
        y = (t(a.real, type=2, axis=axis) + 1j * t(a.imag, type=2, axis=axis)) / (2 * n)
        idx = [slice(None)] * 3
        idx[axis] = n - 1 if kind == "S" else 0
        y[tuple(idx)] *= 0.5
        return y

    a = f.astype(np.complex128)
    if basis[2] == "F":
        a = np.fft.rfft(f, axis=2) / nz
    else:
        a = sc_axis(a, 2, basis[2])
    a = np.fft.fft(a, axis=1) / ny if basis[1] == "F" else sc_axis(a, 1, basis[1])
    a = np.fft.fft(a, axis=0) / nx if basis[0] == "F" else sc_axis(a, 0, basis[0])
    got = oracle_mod.transform3(f, basis)
    assert got.shape == a.shape
    assert np.max(np.abs(got - a)) < 1e-15 * 8
    assert np.max(np.abs(oracle_mod.itransform3(got, nz, basis) - f)) < 1e-13


def test_sss_single_mode_closed_form(oracle_mod):
    # u_z of the all-free-slip basis: 8 cos(kx x) cos(ky y) sin(kz z) -> one coefficient
    n = 16
    X, Y, Z = np.meshgrid(_s(n), _s(n), _s(n), indexing="ij")
    f = 8 * np.cos(2 * X) * np.cos(5 * Y) * np.sin(3 * Z)
    got = oracle_mod.transform3(f, "CCS")
    want = np.zeros((n, n, n))
    want[2, 5, 2] = 1.0
    assert np.max(np.abs(got - want)) < 1e-14


def test_sff_single_mode_closed_form(oracle_mod):
    # 2 sin(kx x) on the free-slip axis times a Fourier mode exp(i(ky y + kz z)) + c.c.
    nx, ny, nz = 8, 8, 16
    y = 2 * np.pi * np.arange(ny) / ny
    z = 2 * np.pi * np.arange(nz) / nz
    X, Y, Z = np.meshgrid(_s(nx), y, z, indexing="ij")
    f = 2 * np.sin(3 * X) * 2 * np.cos(2 * Y + 5 * Z)
    got = oracle_mod.transform3(f, "SFF")
    want = np.zeros((nx, ny, nz // 2 + 1), dtype=complex)
    want[2, 2, 5] = 1.0
    assert np.max(np.abs(got - want)) < 1e-14


def test_bad_bases_rejected(oracle_mod):
    f = np.zeros((4, 4, 4))
    for bad in ("FSF", "FFS", "SFS", [0, 0, 3]):
        with pytest.raises(Exception):
            oracle_mod.transform3(f, bad)


@pytest.mark.parametrize("basis", ["SFF", "SSF", "CCS", "FFF"])
def test_single_coefficient_matches_full_transform(oracle_mod, basis):
    f = synth.uniform_pm1(5, 0, (8, 16, 8))
    full = oracle_mod.transform3(f.astype(np.float64), basis)
    for a, b, c in ((0, 0, 0), (3, 5, 2), (7, 15, full.shape[2] - 1), (1, 9, 4)):
        got = oracle_mod.transform3_coeff(f, basis, a, b, c)
        assert abs(got - full[a, b, c]) < 1e-15
