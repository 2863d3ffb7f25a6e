"""Convection on the periodic cube (FFF, Sec. 2.2, Eqs. (12)-(13)) on grids of
3 * 2^m points, the paper's XC40 convection sizes (Sec. 7): the right-hand
side runs through the plan's transforms (one radix-3 step over power-of-two
sub-lines per 1D pass) with u x omega and u theta formed pointwise in real
space, then the per-mode update of the fused path.  Compared with the FP64
oracle on the same complex64 inputs, relative L2 <= 1e-5 as for the
power-of-two solver.  The 768^3 case uses a band-limited state (|k_i| <= 85),
whose right-hand side is the same set of coefficients on a 768^3 and a 512^3
grid (products reach |k_i| <= 170, alias-free on both).
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


def _kvec(n):
    a = np.arange(n)
    k = np.where(2 * a < n, a, a - n)
    return np.meshgrid(k, k, np.arange(n // 2 + 1), indexing="ij")


def _kept(n):
    KX, KY, KZ = _kvec(n)
    return (3 * np.abs(KX) < n) & (3 * np.abs(KY) < n) & (3 * np.abs(KZ) < n)


def _state(oracle_mod, n, seed, k0=2.0):
    u = oracle_mod.ic_random(synth.normal_fields(seed, 3, (n, n, n)), k0=k0, E0=0.5)
    th = np.fft.rfftn(synth.normal(seed + 1, 0, (n, n, n)).astype(np.float64)) / n**3
    KX, KY, KZ = _kvec(n)
    th = np.where(_kept(n), th * np.exp(-(KX**2 + KY**2 + KZ**2) / (2 * k0 * k0)), 0.0)
    th[0, 0, 0] = 0.0
    th *= np.sqrt(0.1 / (0.5 * np.sum(np.where(KZ == 0, 1.0, 2.0) * np.abs(th) ** 2)))  # 1/2 <theta^2> = 0.1
    return np.concatenate([u, th[None]], axis=0).astype(np.complex64)


def _rhs(fk, plan, s):
    sd = to_dev_c64(s)
    od = to_dev_c64(np.zeros_like(s))
    fk.tarang_rbc_rhs(plan, sd.data_ptr(), od.data_ptr(), stream())
    sync()
    return from_dev_c64(od)


@pytest.mark.parametrize("n", [12, 24, 48, 96])
def test_rbc_rhs_matches_oracle(fk, oracle_mod, n):
    s = _state(oracle_mod, n, 60 + n, k0=min(2.0, n / 8))
    plan = fk.fftk_plan_create(n, n, n)
    try:
        got = _rhs(fk, plan, s)
    finally:
        fk.fftk_plan_destroy(plan)
    want = oracle_mod.rbc_rhs(s.astype(np.complex128))
    assert rel_l2(got[:3], want[:3]) < 1e-5
    assert rel_l2(got[3], want[3]) < 1e-5
    assert not np.any(got[:, ~_kept(n)])


@pytest.mark.parametrize("scheme", [0, 1])
def test_rbc_steps_match_oracle(fk, oracle_mod, scheme):
    n, Ra, Pr, dt, steps = 48, 1e5, 1.0, 2e-3, 8
    s = _state(oracle_mod, n, 70 + scheme)
    plan = fk.fftk_plan_create(n, n, n)
    try:
        sd = to_dev_c64(s)
        fk.tarang_rbc_step(plan, sd.data_ptr(), Ra, Pr, dt, steps, scheme, stream())
        sync()
        got = from_dev_c64(sd)
    finally:
        fk.fftk_plan_destroy(plan)
    want = oracle_mod.rbc_step(s.astype(np.complex128), Ra, Pr, dt, steps, scheme)
    assert rel_l2(got[:3], want[:3]) < 1e-5
    assert rel_l2(got[3], want[3]) < 1e-5


def test_rbc_plane_wave_grows_as_the_exact_solution(fk):
    n, kx, kz, A, B = 48, 2, 1, 0.3, -0.7
    Ra, Pr, dt, steps = 1e4, 0.7, 1e-2, 300
    nu, kappa = np.sqrt(Pr / Ra), 1 / np.sqrt(Ra * Pr)
    k2, sig = kx * kx + kz * kz, kx / np.hypot(kx, kz)
    lam, V = np.linalg.eigh(np.array([[-nu * k2, sig], [sig, -kappa * k2]]))
    A1, B1 = V @ (np.exp(lam * dt * steps) * (V.T @ np.array([A, B])))
    g = 2 * np.pi * np.arange(n) / n
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    e = np.array([-kx * kz, 0.0, kx * kx]) / (kx * np.hypot(kx, kz))

    def wave(a, b):
        c = np.cos(kx * X + kz * Z)
        return np.fft.rfftn(np.stack([a * e[0] * c, a * e[1] * c, a * e[2] * c, b * c]), axes=(1, 2, 3)) / n**3

    plan = fk.fftk_plan_create(n, n, n)
    try:
        sd = to_dev_c64(wave(A, B))
        fk.tarang_rbc_step(plan, sd.data_ptr(), Ra, Pr, dt, steps, fk.TARANG_RK4, stream())
        sync()
        got = from_dev_c64(sd)
    finally:
        fk.fftk_plan_destroy(plan)
    want = wave(A1, B1)
    assert np.max(np.abs(got - want)) < 3e-5 * np.max(np.abs(want))
    assert abs(B1) > 1.5 * abs(B)


def test_rbc_transfer_matches_oracle(fk, oracle_mod):
    n = 48
    s = _state(oracle_mod, n, 80)
    plan = fk.fftk_plan_create(n, n, n)
    try:
        sd = to_dev_c64(s)
        (tu, Tu, Pu), (tt, Tt, Pt) = fk.tarang_rbc_transfer(plan, sd.data_ptr(), stream())
    finally:
        fk.fftk_plan_destroy(plan)
    s64 = s.astype(np.complex128)
    N = oracle_mod.rbc_rhs(s64)
    z = np.zeros_like(s64[0])

    def ts(a, b):
        return oracle_mod.transfer_spectrum(np.stack([a, z, z]), np.stack([b, z, z]))

    Tu_o = oracle_mod.transfer_spectrum(s64[:3], N[:3]) - ts(s64[2], s64[3])
    Tt_o = ts(s64[3], N[3]) - ts(s64[3], s64[2])
    for got, want in ((np.array(Tu), Tu_o), (np.array(Tt), Tt_o)):
        assert np.max(np.abs(want)) > 1e-4
        assert np.max(np.abs(got - want)) < 1e-5 * np.sum(np.abs(want))
    assert abs(tu) < 1e-5 * np.sum(np.abs(Tu)) and abs(tt) < 1e-5 * np.sum(np.abs(Tt))


def test_plates_need_power_of_two_axes(fk, oracle_mod):
    n = 48
    s = _state(oracle_mod, n, 90)
    plan = fk.fftk_plan_create(n, n, n)
    try:
        sd = to_dev_c64(s)
        od = to_dev_c64(np.zeros_like(s))
        with pytest.raises(fk.FFTKError) as e:
            fk.tarang_rbc_rhs(plan, sd.data_ptr(), od.data_ptr(), stream(), basis=fk.TARANG_RBC_SFF)
        assert e.value.status == fk.FFTK_ERR_UNSUPPORTED_SIZE
        with pytest.raises(fk.FFTKError) as e:
            fk.tarang_rbc_step(plan, sd.data_ptr(), 1e5, 1.0, 1e-3, 1, fk.TARANG_RK4, stream(),
                               basis=fk.TARANG_RBC_SFF)
        assert e.value.status == fk.FFTK_ERR_UNSUPPORTED_SIZE
    finally:
        fk.fftk_plan_destroy(plan)


def _embed(s, N):
    n = s.shape[1]
    a = np.arange(n)
    a = a[2 * a != n]
    big = np.where(2 * a < n, a, a - n + N)
    out = np.zeros((s.shape[0], N, N, N // 2 + 1), dtype=s.dtype)
    for f in range(s.shape[0]):
        out[f][np.ix_(big, big, np.arange(n // 2 + 1))] = s[f][np.ix_(a, a, np.arange(n // 2 + 1))]
    return out


def test_rbc_rhs_768_band_limited_matches_oracle_at_512(fk, oracle_mod):
    s256 = _state(oracle_mod, 256, 100, k0=16.0)
    No = oracle_mod.rbc_rhs(_embed(s256, 512).astype(np.complex128))
    s768 = _embed(s256, 768)
    plan = fk.fftk_plan_create(768, 768, 768)
    try:
        Ng = _rhs(fk, plan, s768)
    finally:
        fk.fftk_plan_destroy(plan)
    del s768
    a = np.arange(512)
    rows = np.where(2 * a < 512, a, a - 512 + 768)  # the 512^3 grid's rows inside the 768^3 one
    sub = np.stack([Ng[f][np.ix_(rows, rows, np.arange(257))] for f in range(4)])
    rel_u, rel_t = rel_l2(sub[:3], No[:3]), rel_l2(sub[3], No[3])
    inside = np.zeros(768, dtype=bool)
    inside[rows] = True
    out = 0.0
    for f in range(4):
        for i in range(768):
            row = Ng[f, i].astype(np.complex128)
            if inside[i]:
                out += float(np.sum(np.abs(row[~inside, :]) ** 2) + np.sum(np.abs(row[inside, 257:]) ** 2))
            else:
                out += float(np.sum(np.abs(row) ** 2))
    rel_out = np.sqrt(out) / np.linalg.norm(No.ravel())
    print(f"\nMEASURED rbc rhs768 band-limited rel_l2 u {rel_u:.3e} theta {rel_t:.3e} outside {rel_out:.3e}")
    assert rel_u < 1e-5 and rel_t < 1e-5 and rel_out < 1e-5
