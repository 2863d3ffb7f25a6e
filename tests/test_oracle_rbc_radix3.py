"""Pins for the oracle's Rayleigh-Benard solver (Sec. 2.2, Eqs. (12)-(13),
FFF basis) on cubic grids of 3 * 2^m points, the sizes of the paper's
convection runs on the Cray XC40 (Sec. 7).  The operator's code is the same
as on 2^m grids; only its 1D transforms take 3 * 2^m-point lines by the DFT's
definition.  Closed forms (a plane wave with u perpendicular to k, whose
amplitude and temperature follow a 2x2 linear system), the Navier-Stokes
limit, exact invariants of the advective terms, the advective form of the
temperature term, and a band-limited state whose right-hand side is the same
on a 24^3 and a 32^3 grid.
"""
import numpy as np
import pytest

import synth

N3 = 24  # 3 * 2^3


def _grid(n):
    g = 2 * np.pi * np.arange(n) / n
    return np.meshgrid(g, g, g, indexing="ij")


def _fwd(f):
    return np.fft.rfftn(f, axes=(-3, -2, -1)) / f.shape[-1] ** 3


def _inv(F, n):
    return np.fft.irfftn(F * n**3, s=(n, n, n), axes=(-3, -2, -1))


def _kvec(n):
    a = np.arange(n)
    k = np.where(2 * a < n, a, a - n)
    return np.meshgrid(k, k, np.arange(n // 2 + 1), indexing="ij")


def _kept(n):
    KX, KY, KZ = _kvec(n)
    return (3 * np.abs(KX) < n) & (3 * np.abs(KY) < n) & (3 * np.abs(KZ) < n)


def _state(oracle_mod, n, seed, k0=2.0):
    u = oracle_mod.ic_random(synth.normal_fields(seed, 3, (n, n, n)), k0=k0, E0=0.5)
    th = _fwd(synth.normal(seed + 1, 0, (n, n, n)).astype(np.float64))
    KX, KY, KZ = _kvec(n)
    th = np.where(_kept(n), th * np.exp(-(KX**2 + KY**2 + KZ**2) / (2 * k0 * k0)), 0.0)
    th[0, 0, 0] = 0.0
    return np.concatenate([u, th[None]], axis=0)


def _plane_wave(n, kx, kz, A, B):
    X, Y, Z = _grid(n)
    e = np.array([-kx * kz, 0.0, kx * kx]) / (kx * np.hypot(kx, kz))
    c = np.cos(kx * X + kz * Z)
    return _fwd(np.stack([A * e[0] * c, A * e[1] * c, A * e[2] * c, B * c])), e


def test_plane_wave_rhs_is_the_linear_coupling(oracle_mod):
    kx, kz, A, B = 2, 3, 0.3, -0.7
    s, e = _plane_wave(N3, kx, kz, A, B)
    N = oracle_mod.rbc_rhs(s)
    sig = kx / np.hypot(kx, kz)
    assert np.max(np.abs(N[:3] - np.stack([sig * e[i] * s[3] for i in range(3)]))) < 1e-15
    assert np.max(np.abs(N[3] - s[2])) < 1e-15


@pytest.mark.parametrize("scheme,tol", [(1, 1e-9), (0, 1e-4)])
def test_plane_wave_follows_exact_linear_solution(oracle_mod, scheme, tol):
    kx, kz, A, B = 2, 1, 0.3, -0.7
    Ra, Pr, dt, steps = 1e4, 0.7, 1e-2, 300
    nu, kappa = np.sqrt(Pr / Ra), 1 / np.sqrt(Ra * Pr)
    k2, sig = kx * kx + kz * kz, kx / np.hypot(kx, kz)
    lam, V = np.linalg.eigh(np.array([[-nu * k2, sig], [sig, -kappa * k2]]))
    A1, B1 = V @ (np.exp(lam * dt * steps) * (V.T @ np.array([A, B])))
    s0, _ = _plane_wave(N3, kx, kz, A, B)
    want, _ = _plane_wave(N3, kx, kz, A1, B1)
    got = oracle_mod.rbc_step(s0, Ra, Pr, dt, steps, scheme)
    assert np.max(np.abs(got - want)) < tol * np.max(np.abs(want))
    assert abs(B1) > 1.5 * abs(B)  # the mode grows: the test is not trivially satisfied


def test_without_temperature_velocity_term_is_navier_stokes(oracle_mod):
    s = _state(oracle_mod, N3, 3)
    s[3] = 0
    N = oracle_mod.rbc_rhs(s)
    assert np.max(np.abs(N[:3] - oracle_mod.ns_rhs(s[:3]))) < 1e-15
    assert np.max(np.abs(N[3] - s[2])) < 1e-15


def test_advection_conserves_both_energies(oracle_mod):
    s = _state(oracle_mod, N3, 4)
    N = oracle_mod.rbc_rhs(s)
    KX, KY, KZ = _kvec(N3)
    w = np.where((KZ == 0) | (2 * KZ == N3), 1.0, 2.0)
    k2 = np.maximum(KX**2 + KY**2 + KZ**2, 1)
    th = s[3]
    buoy = np.stack([-KX * KZ * th / k2, -KY * KZ * th / k2, th - KZ * KZ * th / k2])
    nl_u, nl_t = N[:3] - buoy, N[3] - s[2]
    scale_u = np.sum(w * np.abs(s[:3]) * np.abs(nl_u))
    scale_t = np.sum(w * np.abs(th) * np.abs(nl_t))
    assert scale_u > 1e-3 and scale_t > 1e-3
    assert abs(np.sum(w * np.real(np.conj(s[:3]) * nl_u))) < 1e-13 * scale_u
    assert abs(np.sum(w * np.real(np.conj(th) * nl_t))) < 1e-13 * scale_t


def test_temperature_advective_form_equals_divergence_form(oracle_mod):
    s = _state(oracle_mod, N3, 5)
    N = oracle_mod.rbc_rhs(s)
    KX, KY, KZ = _kvec(N3)
    ur = _inv(s[:3], N3)
    grad = [_inv(1j * K * s[3], N3) for K in (KX, KY, KZ)]
    adv = _fwd(-(ur[0] * grad[0] + ur[1] * grad[1] + ur[2] * grad[2]))
    want = np.where(_kept(N3), adv + s[2], 0.0)
    assert np.max(np.abs(N[3] - want)) < 1e-14 * np.max(np.abs(want))


def test_band_limited_state_same_on_3x2m_and_power_of_two_grids(oracle_mod):
    # |k_i| <= 7 (the 2/3 set of 24^3): products reach |k_i| <= 14, whose
    # aliases on 24^3 land at |k_i| >= 10; on 32^3 nothing aliases onto
    # |k_i| <= 10.  So both grids give the same coefficients on |k_i| <= 7.
    s24 = _state(oracle_mod, N3, 6, k0=3.0)
    a = np.arange(N3)
    a = a[2 * a != N3]
    big = np.where(2 * a < N3, a, a - N3 + 32)
    s32 = np.zeros((4, 32, 32, 17), dtype=complex)
    for f in range(4):
        s32[f][np.ix_(big, big, np.arange(13))] = s24[f][np.ix_(a, a, np.arange(13))]
    N24, N32 = oracle_mod.rbc_rhs(s24), oracle_mod.rbc_rhs(s32)
    k24 = np.where(2 * a < N3, a, a - N3)
    sel = np.abs(k24) <= 7
    sub = np.stack([N32[f][np.ix_(big[sel], big[sel], np.arange(8))] for f in range(4)])
    ref = np.stack([N24[f][np.ix_(a[sel], a[sel], np.arange(8))] for f in range(4)])
    assert np.max(np.abs(sub - ref)) < 1e-14 * np.max(np.abs(ref)) * 10
    assert np.max(np.abs(N32[:, :, :, 8:11])) > 1e-6 * np.max(np.abs(N32))
