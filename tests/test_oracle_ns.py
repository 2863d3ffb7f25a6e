"""Pins for the oracle's Navier-Stokes operator and time stepper (Sec. 2.2,
Eqs. (7)-(8); 2/3 rule; RK2 with a viscous integrating factor).

Closed forms (Taylor-Green, ABC, a shear pair with a known nonlinear term),
exact invariants (zero energy transfer, solenoidality), an independent second
formulation (divergence form) and the time stepper's order of accuracy.
"""
import numpy as np
import pytest

import synth


def _grid(n):
    g = 2 * np.pi * np.arange(n) / n
    return np.meshgrid(g, g, g, indexing="ij")


def _np_rfft3(f):
    return np.fft.rfftn(f, axes=(-3, -2, -1)) / f.shape[-1] ** 3


def _kvec(n):
    a = np.arange(n)
    kx = np.where(2 * a < n, a, a - n)
    kz = np.arange(n // 2 + 1)
    return np.meshgrid(kx, kx, kz, indexing="ij")


def _random_uhat(oracle_mod, n, seed=0, k0=2.0):
    return oracle_mod.ic_random(synth.normal_fields(seed, 3, (n, n, n)), k0=k0, E0=0.5)


def test_taylor_green_has_zero_nonlinear_term(oracle_mod):
    # u x omega = -grad(sin^2 x sin^2 y) for Taylor-Green: projected away
    n = 16
    u = oracle_mod.ic_taylor_green(n)
    N = oracle_mod.ns_rhs(u)
    assert np.max(np.abs(N)) < 1e-15
    assert abs(oracle_mod.diag(u)[0] - 0.25) < 1e-15


def test_abc_beltrami_has_zero_nonlinear_term(oracle_mod):
    n = 16
    u = oracle_mod.ic_abc(n)
    N = oracle_mod.ns_rhs(u)
    assert np.max(np.abs(N)) < 1e-14


def test_shear_pair_closed_form(oracle_mod):
    # u = (sin y, 0, sin x): (u.grad)u = (0, 0, sin y cos x) is solenoidal and
    # not a gradient, so the projected nonlinear term is N = (0, 0, -cos x sin y).
    n = 16
    X, Y, Z = _grid(n)
    ur = np.stack([np.sin(Y), 0 * X, np.sin(X)])
    u = oracle_mod.rfft3(ur)
    N = oracle_mod.ns_rhs(u)
    want = _np_rfft3(np.stack([0 * X, 0 * X, -np.cos(X) * np.sin(Y)]))
    assert np.max(np.abs(N - want)) < 1e-15
    # the divergence form gives the same
    assert np.max(np.abs(oracle_mod.ns_rhs_divergence(u) - want)) < 1e-15


@pytest.mark.parametrize("n", [8, 16])
def test_rotational_equals_divergence_form(oracle_mod, n):
    # On the 2/3-truncated set both forms are alias-free and differ by a gradient
    u = _random_uhat(oracle_mod, n, seed=1, k0=3.0)
    Nr = oracle_mod.ns_rhs(u)
    Nd = oracle_mod.ns_rhs_divergence(u)
    scale = np.max(np.abs(Nd))
    assert scale > 1e-3
    assert np.max(np.abs(Nr - Nd)) < 1e-13 * scale


def test_invariants_transfer_solenoidal_dealiased(oracle_mod):
    n = 16
    u = _random_uhat(oracle_mod, n, seed=2, k0=3.0)
    N = oracle_mod.ns_rhs(u)
    scale = np.sqrt(np.sum(np.abs(N) ** 2) * np.sum(np.abs(u) ** 2))
    assert abs(oracle_mod.transfer(u, N)) < 1e-14 * scale
    KX, KY, KZ = _kvec(n)
    assert np.max(np.abs(KX * N[0] + KY * N[1] + KZ * N[2])) < 1e-14 * np.max(np.abs(N)) * n
    keep = (3 * np.abs(KX) < n) & (3 * np.abs(KY) < n) & (3 * np.abs(KZ) < n)
    assert np.all(N[:, ~keep] == 0)


def test_translation_equivariance(oracle_mod):
    n = 16
    u = _random_uhat(oracle_mod, n, seed=3, k0=3.0)
    KX, KY, KZ = _kvec(n)
    ph = np.exp(-2j * np.pi * (3 * KX + 5 * KY + 1 * KZ) / n)
    Ns = oracle_mod.ns_rhs(u * ph)
    assert np.max(np.abs(Ns - oracle_mod.ns_rhs(u) * ph)) < 1e-14 * np.max(np.abs(Ns))


def test_forcing_injects_exactly_eps(oracle_mod):
    # constant-power forcing f = eps u / (2 E_f) on 1 <= |k|^2 <= 4 adds exactly eps
    # to dE/dt; the nonlinear part adds nothing.
    n = 16
    u = _random_uhat(oracle_mod, n, seed=4, k0=2.0)
    N = oracle_mod.ns_rhs(u, force_eps=0.1, force_k2=(1, 4))
    assert abs(oracle_mod.transfer(u, N) - 0.1) < 1e-14


def test_taylor_green_exact_decay(oracle_mod):
    # With N = 0 the integrating factor is exact for any dt: u(t) = u(0) exp(-2 nu t)
    n, nu, dt, steps = 16, 0.01, 1e-3, 20
    u0 = oracle_mod.ic_taylor_green(n)
    u = oracle_mod.ns_step(u0, nu, dt, steps)
    t = steps * dt
    assert np.max(np.abs(u - u0 * np.exp(-2 * nu * t))) < 1e-15
    assert abs(oracle_mod.diag(u)[0] - 0.25 * np.exp(-4 * nu * t)) < 1e-15


def test_abc_exact_decay(oracle_mod):
    n, nu, dt, steps = 16, 0.05, 0.01, 10
    u0 = oracle_mod.ic_abc(n)
    E0 = oracle_mod.diag(u0)[0]
    u = oracle_mod.ns_step(u0, nu, dt, steps)
    assert abs(oracle_mod.diag(u)[0] - E0 * np.exp(-2 * nu * steps * dt)) < 1e-14


def test_inviscid_energy_drift_is_third_order(oracle_mod):
    # Heun on an energy-conserving system: the per-step amplification
    # |1 + z + z^2/2|^2 = 1 + |z|^4/4 for imaginary z gives an energy error of
    # O(dt^4) per step, O(dt^3) over a fixed time: halving dt divides it by 8.
    n, T = 16, 0.2
    u0 = _random_uhat(oracle_mod, n, seed=0, k0=2.0)
    E0 = oracle_mod.diag(u0)[0]
    d = [oracle_mod.diag(oracle_mod.ns_step(u0, 0.0, dt, int(round(T / dt))))[0] - E0 for dt in (0.02, 0.01)]
    assert d[0] > 0 and d[1] > 0
    assert 8 * 0.9 < d[0] / d[1] < 8 * 1.1
    assert d[1] < 1e-5 * E0


def test_dissipation_is_minus_dEdt(oracle_mod):
    # unforced: dE/dt = -eps; centred difference over one small step
    n, nu, dt = 16, 0.02, 1e-3
    u0 = _random_uhat(oracle_mod, n, seed=5, k0=3.0)
    E0, eps0, _ = oracle_mod.diag(u0, nu)
    u1 = oracle_mod.ns_step(u0, nu, dt, 1)
    E1, eps1, _ = oracle_mod.diag(u1, nu)
    dEdt = (E1 - E0) / dt
    assert abs(dEdt + 0.5 * (eps0 + eps1)) < 1e-4 * eps0


def test_spectrum_sums_to_energy(oracle_mod):
    n = 16
    u = _random_uhat(oracle_mod, n, seed=6, k0=3.0)
    E, eps, EK = oracle_mod.diag(u, 0.01)
    assert abs(EK.sum() - E) < 1e-15
    # eps = 2 nu sum_K K^2 E(K) only approximately (shells round |k|), but
    # eps = nu sum w |k|^2 |u|^2 exactly: recompute with the closed weights
    KX, KY, KZ = _kvec(n)
    w = np.where((KZ == 0) | (2 * KZ == n), 1.0, 2.0)
    k2 = KX**2 + KY**2 + KZ**2
    assert abs(eps - 0.01 * np.sum(w * k2 * np.sum(np.abs(u) ** 2, axis=0))) < 1e-13 * eps


def test_random_ic_properties(oracle_mod):
    n, k0 = 32, 4.0
    u = oracle_mod.ic_random(synth.normal_fields(0, 3, (n, n, n)), k0=k0, E0=0.5)
    E, _, EK = oracle_mod.diag(u)
    assert abs(E - 0.5) < 1e-14
    K = np.arange(EK.size, dtype=np.float64)
    target = K**4 * np.exp(-2 * (K / k0) ** 2)
    present = EK > 0
    assert not present[0]
    ratio = EK[present] / target[present]
    assert np.max(np.abs(ratio / ratio[0] - 1)) < 1e-12
    KX, KY, KZ = _kvec(n)
    assert np.max(np.abs(KX * u[0] + KY * u[1] + KZ * u[2])) < 1e-15
    keep = (3 * np.abs(KX) < n) & (3 * np.abs(KY) < n) & (3 * np.abs(KZ) < n)
    assert np.all(u[:, ~keep] == 0)
    # exactly Hermitian on the k_z = 0 plane
    P = u[:, :, :, 0]
    Pm = np.conj(P[:, (-np.arange(n)) % n][:, :, (-np.arange(n)) % n])
    assert np.max(np.abs(P - Pm)) == 0.0


def test_diag_energy_is_parseval_on_untruncated_field(oracle_mod):
    # E = 1/2 <|u|^2> over the grid, including the k_z = N/2 plane (weight 1)
    n = 8
    rng = np.random.default_rng(7)
    ur = rng.standard_normal((3, n, n, n))
    u = oracle_mod.rfft3(ur)
    assert np.max(np.abs(u[:, :, :, n // 2])) > 0.01
    E = oracle_mod.diag(u)[0]
    assert abs(E - 0.5 * np.mean(np.sum(ur**2, axis=0))) < 1e-14


def _shell_index(n):
    KX, KY, KZ = _kvec(n)
    return np.floor(np.sqrt(KX**2 + KY**2 + KZ**2) + 0.5).astype(int)


def test_transfer_spectrum_is_shell_filtered_power(oracle_mod):
    # Parseval per shell: T(K) = <u_K . N> over the box, u_K the real field of
    # the modes of shell K, computed here on the full complex spectrum (numpy
    # FFT, no Hermitian weights) instead of the half spectrum with w = 1 or 2.
    n = 16
    u = _random_uhat(oracle_mod, n, seed=5, k0=3.0)
    N = oracle_mod.ns_rhs(u)
    T = oracle_mod.transfer_spectrum(u, N)
    ur = np.fft.irfftn(u * n**3, s=(n, n, n), axes=(-3, -2, -1))
    Nr = np.fft.irfftn(N * n**3, s=(n, n, n), axes=(-3, -2, -1))
    U = np.fft.fftn(ur, axes=(-3, -2, -1)) / n**3
    a = np.arange(n)
    k = np.where(2 * a < n, a, a - n)
    KX, KY, KZ = np.meshgrid(k, k, k, indexing="ij")
    shell = np.floor(np.sqrt(KX**2 + KY**2 + KZ**2) + 0.5).astype(int)
    want = np.zeros_like(T)
    for K in range(len(T)):
        uK = np.real(np.fft.ifftn(np.where(shell == K, U, 0), axes=(-3, -2, -1))) * n**3
        want[K] = np.mean(np.sum(uK * Nr, axis=0))
    scale = np.max(np.abs(want))
    assert scale > 1e-4
    assert np.max(np.abs(T - want)) < 1e-13 * scale


def test_transfer_spectrum_conserves_and_matches_total(oracle_mod):
    # the nonlinear term only moves energy between shells: sum_K T(K) = 0,
    # while the individual shells are far from zero
    n = 16
    u = _random_uhat(oracle_mod, n, seed=6, k0=3.0)
    N = oracle_mod.ns_rhs(u)
    T = oracle_mod.transfer_spectrum(u, N)
    assert np.max(np.abs(T)) > 1e-3
    assert abs(T.sum()) < 1e-14 * np.sum(np.abs(T))
    flux = -np.cumsum(T)
    assert abs(flux[-1]) < 1e-14 * np.sum(np.abs(T))


def test_transfer_spectrum_of_forcing_is_eps_in_forced_shell(oracle_mod):
    # the constant-power forcing on 1 <= |k|^2 <= 2 (exactly shell K = 1) adds
    # eps to T(1) and nothing elsewhere
    n, eps = 16, 0.1
    u = _random_uhat(oracle_mod, n, seed=7, k0=2.0)
    T0 = oracle_mod.transfer_spectrum(u, oracle_mod.ns_rhs(u))
    Tf = oracle_mod.transfer_spectrum(u, oracle_mod.ns_rhs(u, force_eps=eps, force_k2=(1, 2)))
    d = Tf - T0
    assert abs(d[1] - eps) < 1e-14
    assert np.max(np.abs(np.delete(d, 1))) < 1e-15


def test_transfer_spectrum_drops_shells_beyond_kmax(oracle_mod):
    n = 16
    u = _random_uhat(oracle_mod, n, seed=8, k0=3.0)
    N = oracle_mod.ns_rhs(u)
    T = oracle_mod.transfer_spectrum(u, N)
    assert np.array_equal(oracle_mod.transfer_spectrum(u, N, kmax=5), T[:6])


def _full_spectrum(uhat, n):
    # the full complex spectrum of the real field (numpy FFT)
    ur = np.fft.irfftn(uhat * n**3, s=(n, n, n), axes=(-3, -2, -1))
    return np.fft.fftn(ur, axes=(-3, -2, -1)) / n**3


def test_shell_transfer_matches_triad_sum(oracle_mod):
    # mode-to-mode form: T[r, g] = sum_{k in r} sum_{p in g} Im[(k . u(k - p)) (conj(u(k)) . u(p))],
    # summed here over all triads of the full spectrum by brute force
    n = 16
    u = _random_uhat(oracle_mod, n, seed=9, k0=2.0)
    bounds = [0, 1, 2, 3, 4, 6, 9]
    T = oracle_mod.shell_transfer(u, bounds)
    U = _full_spectrum(u, n)
    a = np.arange(n)
    k1 = np.where(2 * a < n, a, a - n)
    KX, KY, KZ = np.meshgrid(k1, k1, k1, indexing="ij")
    K = np.floor(np.sqrt(KX**2 + KY**2 + KZ**2) + 0.5).astype(int)
    live = np.nonzero(np.max(np.abs(U), axis=0) > 0)
    modes = np.stack(live, axis=1)
    kvec = np.stack([KX[live], KY[live], KZ[live]], axis=1)
    S = len(bounds) - 1
    shell = np.full(len(modes), -1)
    for i in range(S):
        shell[(K[live] >= bounds[i]) & (K[live] < bounds[i + 1])] = i
    want = np.zeros((S, S))
    for ik in range(len(modes)):
        r = shell[ik]
        if r < 0:
            continue
        k = kvec[ik]
        uk = U[:, modes[ik][0], modes[ik][1], modes[ik][2]]
        q = (modes[ik][None, :] - modes) % n  # index of k - p for every p
        uq = U[:, q[:, 0], q[:, 1], q[:, 2]]
        up = U[:, modes[:, 0], modes[:, 1], modes[:, 2]]
        s = np.imag((k @ uq) * (np.conj(uk) @ up))
        for g in range(S):
            want[r, g] += s[shell == g].sum()
    scale = np.max(np.abs(want))
    assert scale > 1e-3
    assert np.max(np.abs(T - want)) < 1e-12 * scale


def test_shell_transfer_antisymmetric_and_sums_to_transfer_spectrum(oracle_mod):
    # T[r, g] = -T[g, r] (u solenoidal); the givers of a receiver add up to its
    # transfer T(K) over the shell; the flux through a bound is the transfer
    # from the shells inside to those outside
    n = 16
    u = _random_uhat(oracle_mod, n, seed=10, k0=3.0)
    kmax = oracle_mod.kmax_shell(n)
    bounds = [0, 2, 3, 4, 5, 6, 8, 10, 12, kmax + 1]
    T = oracle_mod.shell_transfer(u, bounds)
    scale = np.max(np.abs(T))
    assert scale > 1e-3
    assert np.max(np.abs(T + T.T)) < 1e-13 * scale
    TK = oracle_mod.transfer_spectrum(u, oracle_mod.ns_rhs(u))
    rows = np.array([TK[bounds[i]:bounds[i + 1]].sum() for i in range(len(bounds) - 1)])
    assert np.max(np.abs(T.sum(axis=1) - rows)) < 1e-13 * scale
    flux = -np.cumsum(TK)
    for i in range(1, len(bounds) - 1):
        assert abs(T[i:, :i].sum() - flux[bounds[i] - 1]) < 1e-13 * scale


def test_shell_transfer_rejects_bad_bounds(oracle_mod):
    u = _random_uhat(oracle_mod, 8, seed=0)
    with pytest.raises(Exception):
        oracle_mod.shell_transfer(u, [0, 2, 2, 4])


def test_rk4_taylor_green_exact_decay(oracle_mod):
    # N = 0 for Taylor-Green: the integrating factor makes every stage exact
    n, nu, dt, steps = 16, 0.01, 1e-2, 20
    u0 = oracle_mod.ic_taylor_green(n)
    u = oracle_mod.ns_step_rk4(u0, nu, dt, steps)
    assert np.max(np.abs(u - u0 * np.exp(-2 * nu * steps * dt))) < 1e-15


def test_rk4_is_fourth_order(oracle_mod):
    # global error against a fine-step solution falls by 2^4 when dt halves
    # (and by 2^2 for the second-order scheme on the same problem)
    n, nu, T = 16, 0.02, 0.2
    u0 = _random_uhat(oracle_mod, n, seed=11, k0=2.0)
    ref = oracle_mod.ns_step_rk4(u0, nu, T / 64, 64)
    e4 = [np.linalg.norm(oracle_mod.ns_step_rk4(u0, nu, T / s, s) - ref) for s in (4, 8)]
    e2 = [np.linalg.norm(oracle_mod.ns_step(u0, nu, T / s, s) - ref) for s in (8, 16)]
    assert 13.0 < e4[0] / e4[1] < 19.0, e4
    assert 3.3 < e2[0] / e2[1] < 4.7, e2


def test_rk4_matches_rk2_at_small_dt(oracle_mod):
    n, nu, T = 16, 0.01, 0.05
    u0 = _random_uhat(oracle_mod, n, seed=12, k0=2.0)
    a = oracle_mod.ns_step_rk4(u0, nu, T / 10, 10)
    b = oracle_mod.ns_step(u0, nu, T / 200, 200)
    assert np.linalg.norm(a - b) < 1e-6 * np.linalg.norm(a)


def test_rk4_forced_energy_budget(oracle_mod):
    # dE/dt = eps_injected - dissipation: over a short interval with the
    # constant-power forcing, E(T) - E(0) = eps T - int 2 nu Z dt (trapezoid)
    n, nu, dt, steps, eps = 16, 0.02, 2e-3, 10, 0.1
    u0 = _random_uhat(oracle_mod, n, seed=13, k0=2.0)
    E0, d0, _ = oracle_mod.diag(u0, nu)
    u = oracle_mod.ns_step_rk4(u0, nu, dt, steps, force_eps=eps, force_k2=(1, 4))
    E1, d1, _ = oracle_mod.diag(u, nu)
    T = dt * steps
    assert abs((E1 - E0) - (eps * T - 0.5 * (d0 + d1) * T)) < 2e-3 * abs(E1 - E0) + 1e-6
