"""Pins for the oracle's Navier-Stokes operator (Sec. 2.2, Eqs. (7)-(8), 2/3
rule) and time stepper on cubic grids of 3 * 2^m points, the sizes of the
paper's runs on the Cray XC40 (768^3 to 3072^3, Sec. 6-7).  There the
oracle's 1D transforms take each line of 3 * 2^m points by the DFT's
definition instead of the recursive radix-2 FFT; the operator's own code is
the same.  Closed forms (Taylor-Green, ABC, a shear pair), exact invariants,
the divergence form, the exact viscous decay, and the same band-limited field
on a 24^3 and a 32^3 grid (power-of-two transforms), whose right-hand sides
must agree on every mode both grids keep.
"""
import numpy as np

import synth

N3 = 24  # 3 * 2^3


def _grid(n):
    g = 2 * np.pi * np.arange(n) / n
    return np.meshgrid(g, g, g, indexing="ij")


def _kvec(n):
    a = np.arange(n)
    kx = np.where(2 * a < n, a, a - n)
    return np.meshgrid(kx, kx, np.arange(n // 2 + 1), indexing="ij")


def _random(oracle_mod, n, seed=3, k0=3.0):
    return oracle_mod.ic_random(synth.normal_fields(seed, 3, (n, n, n)), k0=k0, E0=0.5)


def test_taylor_green_and_abc_have_zero_nonlinear_term(oracle_mod):
    u = oracle_mod.ic_taylor_green(N3)
    assert np.max(np.abs(oracle_mod.ns_rhs(u))) < 1e-14
    assert abs(oracle_mod.diag(u)[0] - 0.25) < 1e-14
    assert np.max(np.abs(oracle_mod.ns_rhs(oracle_mod.ic_abc(N3)))) < 1e-13


def test_shear_pair_closed_form(oracle_mod):
    # u = (sin y, 0, sin x): the projected nonlinear term is (0, 0, -cos x sin y)
    X, Y, Z = _grid(N3)
    u = oracle_mod.rfft3(np.stack([np.sin(Y), 0 * X, np.sin(X)]))
    want = np.fft.rfftn(np.stack([0 * X, 0 * X, -np.cos(X) * np.sin(Y)]), axes=(1, 2, 3)) / N3**3
    assert np.max(np.abs(oracle_mod.ns_rhs(u) - want)) < 1e-14
    assert np.max(np.abs(oracle_mod.ns_rhs_divergence(u) - want)) < 1e-14


def test_invariants_of_a_random_field(oracle_mod):
    u = _random(oracle_mod, N3)
    N = oracle_mod.ns_rhs(u)
    scale = np.sqrt(np.sum(np.abs(N) ** 2) * np.sum(np.abs(u) ** 2))
    # zero energy transfer (alias-free products of 2/3-truncated fields) and k . N = 0
    assert abs(oracle_mod.transfer(u, N)) < 1e-13 * scale
    KX, KY, KZ = _kvec(N3)
    assert np.max(np.abs(KX * N[0] + KY * N[1] + KZ * N[2])) < 1e-13 * np.max(np.abs(N)) * N3
    # rotational form = divergence form on the kept modes
    assert np.max(np.abs(N - oracle_mod.ns_rhs_divergence(u))) < 1e-13 * np.max(np.abs(N))
    # constant-power forcing injects exactly eps
    Nf = oracle_mod.ns_rhs(u, force_eps=0.1, force_k2=(1, 4))
    assert abs(oracle_mod.transfer(u, Nf) - 0.1) < 1e-12


def _embed(u, N):
    n = u.shape[1]
    a = np.arange(n)
    a = a[2 * a != n]
    big = np.where(2 * a < n, a, a - n + N)
    out = np.zeros((3, N, N, N // 2 + 1), dtype=u.dtype)
    for c in range(3):
        out[c][np.ix_(big, big, np.arange(n // 2 + 1))] = u[c][np.ix_(a, a, np.arange(n // 2 + 1))]
    return out, big


def test_band_limited_field_same_on_3x2m_and_power_of_two_grids(oracle_mod):
    # a field with |k_i| <= 7 (the 2/3 set of 24^3): its products reach
    # |k_i| <= 14, whose aliases on 24^3 fall at |k_i| >= 10, outside the kept
    # |k_i| <= 7; on 32^3 nothing aliases onto |k_i| <= 10.  So on the modes
    # with |k_i| <= 7 both grids give the truncated convolution.
    u24 = _random(oracle_mod, N3, seed=5, k0=4.0)
    u32, big = _embed(u24, 32)
    N24 = oracle_mod.ns_rhs(u24)
    N32 = oracle_mod.ns_rhs(u32)
    a = np.arange(N3)
    keep = np.abs(np.where(2 * a < N3, a, a - N3)) <= 7
    sub = np.stack([N32[c][np.ix_(big[keep[a != N3 // 2]], big[keep[a != N3 // 2]], np.arange(8))]
                    for c in range(3)])
    ref = np.stack([N24[c][np.ix_(a[keep], a[keep], np.arange(8))] for c in range(3)])
    assert np.max(np.abs(sub - ref)) < 1e-14 * np.max(np.abs(ref)) * 10
    # and 32^3 holds more: the products' modes 8 <= |k_i| <= 10 are not zero there
    assert np.max(np.abs(N32)) > 0 and np.max(np.abs(N32[:, :, :, 8:11])) > 1e-6 * np.max(np.abs(N32))


def test_taylor_green_exact_decay_rk2_and_rk4(oracle_mod):
    nu, dt, steps = 0.01, 1e-3, 20
    u0 = oracle_mod.ic_taylor_green(N3)
    want = 0.25 * np.exp(-4 * nu * steps * dt)
    for step in (oracle_mod.ns_step, oracle_mod.ns_step_rk4):
        E = oracle_mod.diag(step(u0, nu, dt, steps))[0]
        assert abs(E - want) < 1e-14


def test_random_initial_field_energy_and_shells(oracle_mod):
    u = _random(oracle_mod, N3, seed=7, k0=2.0)
    E, _, EK = oracle_mod.diag(u)
    assert abs(E - 0.5) < 1e-14
    K = np.arange(len(EK))
    target = K**4.0 * np.exp(-2 * (K / 2.0) ** 2)
    live = EK > 0
    ratio = EK[live] / target[live]
    assert np.max(np.abs(ratio / ratio[0] - 1)) < 1e-12
    KX, KY, KZ = _kvec(N3)
    assert np.max(np.abs(KX * u[0] + KY * u[1] + KZ * u[2])) < 1e-14
