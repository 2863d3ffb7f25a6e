"""Pins for the oracle's Rayleigh-Benard solver (Sec. 2.2, Eqs. (12)-(13),
FFF basis, gravity along z).

A single plane wave with u perpendicular to k has no nonlinear interaction,
so its amplitude and temperature follow a 2x2 linear system exactly (closed
form by the eigenvectors of a symmetric matrix); with theta = 0 the velocity
part is the Navier-Stokes term; advection conserves 1/2 |u|^2 and 1/2 theta^2
on the truncated set; the temperature term in advective form (gradient, then
product) equals the divergence form; RK4 is fourth order.
"""
import numpy as np
import pytest

import synth


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


def _weights(n):
    KX, KY, KZ = _kvec(n)
    return np.where((KZ == 0) | (2 * KZ == n), 1.0, 2.0)


def _random_state(oracle_mod, n, seed):
    u = oracle_mod.ic_random(synth.normal_fields(seed, 3, (n, n, n)), k0=2.0, E0=0.5)
    th = _fwd(synth.normal(seed + 1, 0, (n, n, n)).astype(np.float64))
    KX, KY, KZ = _kvec(n)
    keep = (3 * np.abs(KX) < n) & (3 * np.abs(KY) < n) & (3 * np.abs(KZ) < n)
    th = np.where(keep, th * np.exp(-(KX**2 + KY**2 + KZ**2) / 8.0), 0.0)
    th[0, 0, 0] = 0.0
    return np.concatenate([u, th[None]], axis=0)


def _plane_wave(n, kx, kz, A, B):
    X, Y, Z = _grid(n)
    k = np.hypot(kx, kz)
    e = np.array([-kx * kz, 0.0, kx * kx]) / (kx * k)  # unit vector perpendicular to k in the x-z plane
    c = np.cos(kx * X + kz * Z)
    real = np.stack([A * e[0] * c, A * e[1] * c, A * e[2] * c, B * c])
    return _fwd(real), e


def test_plane_wave_rhs_is_linear(oracle_mod):
    n, kx, kz, A, B = 16, 2, 1, 0.3, -0.7
    s, e = _plane_wave(n, kx, kz, A, B)
    N = oracle_mod.rbc_rhs(s)
    sig = kx / np.hypot(kx, kz)
    # N_u = P[theta z] = sigma theta e, N_theta = u_z = sigma A (in the same mode)
    want_u = np.stack([sig * e[i] * s[3] for i in range(3)])
    assert np.max(np.abs(N[:3] - want_u)) < 1e-15
    assert np.max(np.abs(N[3] - s[2])) < 1e-15


@pytest.mark.parametrize("scheme,tol", [(1, 1e-9), (0, 1e-4)])
def test_plane_wave_follows_exact_linear_solution(oracle_mod, scheme, tol):
    n, kx, kz, A, B = 16, 2, 1, 0.3, -0.7
    Ra, Pr, dt, steps = 1e4, 0.7, 1e-2, 300
    nu, kappa = np.sqrt(Pr / Ra), 1 / np.sqrt(Ra * Pr)
    k2, sig = kx * kx + kz * kz, kx / np.hypot(kx, kz)
    Mx = np.array([[-nu * k2, sig], [sig, -kappa * k2]])
    lam, V = np.linalg.eigh(Mx)
    t = dt * steps
    A1, B1 = V @ (np.exp(lam * t) * (V.T @ np.array([A, B])))
    s0, _ = _plane_wave(n, kx, kz, A, B)
    want, _ = _plane_wave(n, kx, kz, A1, B1)
    got = oracle_mod.rbc_step(s0, Ra, Pr, dt, steps, scheme)
    assert np.max(np.abs(got - want)) < tol * np.max(np.abs(want))
    assert abs(B1) > 1.5 * abs(B)  # the mode grows: the test is not trivially satisfied


def test_without_temperature_velocity_term_is_navier_stokes(oracle_mod):
    n = 16
    s = _random_state(oracle_mod, n, 3)
    s[3] = 0
    N = oracle_mod.rbc_rhs(s)
    assert np.max(np.abs(N[:3] - oracle_mod.ns_rhs(s[:3]))) < 1e-15
    assert np.max(np.abs(N[3] - s[2])) < 1e-15


def test_advection_conserves_both_energies(oracle_mod):
    n = 16
    s = _random_state(oracle_mod, n, 4)
    N = oracle_mod.rbc_rhs(s)
    w = _weights(n)
    KX, KY, KZ = _kvec(n)
    k2 = np.maximum(KX**2 + KY**2 + KZ**2, 1)
    th = s[3]
    buoy = np.stack([-KX * KZ * th / k2, -KY * KZ * th / k2, th - KZ * KZ * th / k2])
    nl_u = N[:3] - buoy
    nl_t = N[3] - s[2]
    scale_u = np.sum(w * np.abs(s[:3]) * np.abs(nl_u))
    scale_t = np.sum(w * np.abs(th) * np.abs(nl_t))
    assert scale_u > 1e-3 and scale_t > 1e-3
    assert abs(np.sum(w * np.real(np.conj(s[:3]) * nl_u))) < 1e-13 * scale_u
    assert abs(np.sum(w * np.real(np.conj(th) * nl_t))) < 1e-13 * scale_t


def test_temperature_advective_form_equals_divergence_form(oracle_mod):
    # -u . grad theta computed by numpy (gradient in Fourier space, product in real space)
    n = 16
    s = _random_state(oracle_mod, n, 5)
    N = oracle_mod.rbc_rhs(s)
    KX, KY, KZ = _kvec(n)
    ur = _inv(s[:3], n)
    grad = [_inv(1j * K * s[3], n) for K in (KX, KY, KZ)]
    adv = _fwd(-(ur[0] * grad[0] + ur[1] * grad[1] + ur[2] * grad[2]))
    keep = (3 * np.abs(KX) < n) & (3 * np.abs(KY) < n) & (3 * np.abs(KZ) < n)
    want = np.where(keep, adv + s[2], 0.0)
    assert np.max(np.abs(N[3] - want)) < 1e-14 * np.max(np.abs(want))


def test_rbc_rk4_is_fourth_order(oracle_mod):
    n, Ra, Pr, T = 16, 1e4, 1.0, 0.2
    s0 = _random_state(oracle_mod, n, 6)
    ref = oracle_mod.rbc_step(s0, Ra, Pr, T / 64, 64, 1)
    e = [np.linalg.norm(oracle_mod.rbc_step(s0, Ra, Pr, T / m, m, 1) - ref) for m in (4, 8)]
    assert 13.0 < e[0] / e[1] < 19.0, e
