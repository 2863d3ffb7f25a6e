"""Pins for the oracle's closure pieces: box filter, spectral gradient,
invariants, eigenframe, MLP (forward, backward, Adam) and the SGS force."""
import numpy as np
import pytest

import synth

RNG = np.random.default_rng(2024)


def _grid(n):
    g = 2 * np.pi * np.arange(n) / n
    return np.meshgrid(g, g, g, indexing="ij")


def test_box_filter_constant_and_blockwise_constant(oracle_mod):
    n, f = 16, 4
    u = np.stack([np.full((n, n, n), 1.5), np.full((n, n, n), -2.0), np.zeros((n, n, n))])
    ubar, tau = oracle_mod.box_filter(u, f)
    assert np.allclose(ubar[0], 1.5) and np.allclose(ubar[1], -2.0)
    assert np.max(np.abs(tau)) < 1e-15
    blocks = RNG.standard_normal((3, n // f, n // f, n // f))
    u = np.repeat(np.repeat(np.repeat(blocks, f, 1), f, 2), f, 3)
    ubar, tau = oracle_mod.box_filter(u, f)
    assert np.max(np.abs(ubar - blocks)) < 1e-13
    assert np.max(np.abs(tau)) < 1e-13


def test_box_filter_of_a_mode_with_the_block_wavelength(oracle_mod):
    # cos of a wave with exactly one period per block averages to 0 over the
    # block; its square averages to 1/2, so tau_xx = 1/2 and tau_xy = 0
    n, f = 32, 8
    X, Y, Z = _grid(n)
    u = np.stack([np.cos(n / f * X), np.ones_like(X), np.zeros_like(X)])
    ubar, tau = oracle_mod.box_filter(u, f)
    assert np.max(np.abs(ubar[0])) < 1e-15
    assert np.max(np.abs(tau[0] - 0.5)) < 1e-15
    assert np.max(np.abs(tau[3])) < 1e-15  # xy: <cos * 1> - 0 * 1


def test_gradient_closed_form(oracle_mod):
    m = 16
    X, Y, Z = _grid(m)
    u = np.stack([np.sin(Y), np.cos(Z), np.sin(2 * X)])
    A = oracle_mod.gradient(u)
    want = np.zeros((9,) + X.shape)
    want[1] = np.cos(Y)           # d u_x / dy
    want[5] = -np.sin(Z)          # d u_y / dz
    want[6] = 2 * np.cos(2 * X)   # d u_z / dx
    assert np.max(np.abs(A - want)) < 1e-13


def test_invariants_against_eigenvalues_and_vorticity(oracle_mod):
    for _ in range(5):
        A = RNG.standard_normal((3, 3))
        inv = oracle_mod.invariants(A.ravel())
        S = 0.5 * (A + A.T)
        lam = np.linalg.eigvalsh(S)
        w = np.array([A[2, 1] - A[1, 2], A[0, 2] - A[2, 0], A[1, 0] - A[0, 1]])  # vorticity
        assert abs(inv[0] - np.sum(lam**2)) < 1e-12
        assert abs(inv[2] - np.sum(lam**3)) < 1e-12
        assert abs(inv[1] + 0.5 * w @ w) < 1e-12  # tr R^2 = -|omega|^2 / 2
        # tr R^2 S = (|w|^2 tr S - w.S.w)/4 * (-1) ... = (w.S.w - |w|^2 tr S) / 4
        assert abs(inv[3] - (w @ S @ w - (w @ w) * np.trace(S)) / 4) < 1e-12
    # pure rotation: only tr R^2 is nonzero
    inv = oracle_mod.invariants(np.array([[0, -3.0, 0], [3.0, 0, 0], [0, 0, 0]]).ravel())
    assert np.allclose(inv, [0, -18.0, 0, 0, 0])


def test_sym_eig3(oracle_mod):
    for _ in range(20):
        M = RNG.standard_normal((3, 3))
        S = M + M.T
        lam, Q = oracle_mod.sym_eig3(S.ravel())
        assert np.allclose(lam, np.sort(np.linalg.eigvalsh(S))[::-1], atol=1e-12)
        assert np.allclose(Q.T @ Q, np.eye(3), atol=1e-12)
        assert np.allclose(Q @ np.diag(lam) @ Q.T, S, atol=1e-12)
        for k in range(3):
            big = np.argmax(np.abs(Q[:, k]))
            assert Q[big, k] > 0


def _random_params(scale=0.3, seed=0):
    r = np.random.default_rng(seed)
    return r.standard_normal(9094) * scale


def test_mlp_forward_closed_form(oracle_mod):
    # with W1 = W2 = W3 = 0 the hidden layers are tanh of their biases
    p = _random_params()
    o = 0
    dims = [5, 64, 64, 64, 6]
    offs = []
    for l in range(4):
        w = o
        b = o + dims[l + 1] * dims[l]
        offs.append((w, b))
        o = b + dims[l + 1]
    assert o == 9094
    for l in range(3):
        w, b = offs[l]
        p[w:b] = 0.0
    x = RNG.standard_normal((7, 5))
    y = oracle_mod.mlp_forward(p, x, bf16_acts=False)
    h3 = np.tanh(p[offs[2][1]:offs[2][1] + 64])
    W4 = p[offs[3][0]:offs[3][1]].reshape(6, 64)
    want = W4 @ h3 + p[offs[3][1]:offs[3][1] + 6]
    assert np.max(np.abs(y - want[None, :])) < 1e-14


def test_mlp_gradient_matches_finite_differences(oracle_mod):
    p = _random_params(0.4, seed=1)
    x = RNG.standard_normal((9, 5))
    t = RNG.standard_normal((9, 6))
    loss, g = oracle_mod.mlp_loss_grad(p, x, t, bf16_acts=False)
    y = oracle_mod.mlp_forward(p, x, bf16_acts=False)
    assert abs(loss - np.mean((y - t) ** 2)) < 1e-15
    h = 1e-6
    idx = np.concatenate([np.arange(0, 9094, 97), [0, 319, 320, 383, 9087, 9093]])
    for i in idx:
        pp = p.copy()
        pp[i] += h
        lp, _ = oracle_mod.mlp_loss_grad(pp, x, t, bf16_acts=False)
        pp[i] -= 2 * h
        lm, _ = oracle_mod.mlp_loss_grad(pp, x, t, bf16_acts=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9


def test_mlp_bf16_rounding_changes_little(oracle_mod):
    p = _random_params(0.3, seed=2)
    x = RNG.standard_normal((32, 5))
    a = oracle_mod.mlp_forward(p, x, bf16_acts=False)
    b = oracle_mod.mlp_forward(p, x, bf16_acts=True)
    rel = np.linalg.norm(a - b) / np.linalg.norm(a)
    assert 1e-5 < rel < 2e-2  # bfloat16 keeps 8 bits: a visible but small change


def test_adam_first_steps_closed_form(oracle_mod):
    # from zero moments with a constant gradient g: every step moves by
    # lr * g / (|g| + eps) (bias corrections cancel exactly)
    n = 11
    p = np.linspace(-1, 1, n)
    p0 = p.copy()
    m = np.zeros(n)
    v = np.zeros(n)
    g = np.linspace(-3, 2, n)
    for step in (1, 2, 3):
        oracle_mod.adam(p, m, v, g, step, lr=1e-3)
    want = p0 - 3 * 1e-3 * g / (np.abs(g) + 1e-8)
    assert np.max(np.abs(p - want)) < 1e-12


def test_sgs_force_closed_form(oracle_mod):
    # tau_xy = tau_yx = sin x, other components 0: s_i = -d_j tau_ij gives
    # s = (-d_y sin x, -d_x sin x, 0) = (0, -cos x, 0), already solenoidal
    n = 16
    X, Y, Z = _grid(n)
    tau = np.zeros((6, n, n, n))
    tau[3] = np.sin(X)
    f = oracle_mod.sgs_force(tau)
    want = np.fft.rfftn(np.stack([0 * X, -np.cos(X), 0 * X]), axes=(1, 2, 3)) / n**3
    assert np.max(np.abs(f - want)) < 1e-15


def test_box_filter_brute_force_random(oracle_mod):
    # block means by reshaping (an independent computation) on a random field
    n, f = 8, 2
    u = RNG.standard_normal((3, n, n, n))
    ubar, tau = oracle_mod.box_filter(u, f)
    m = n // f
    blk = lambda a: a.reshape(m, f, m, f, m, f).mean(axis=(1, 3, 5))
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    for q in range(3):
        assert np.max(np.abs(ubar[q] - blk(u[q]))) < 1e-14
    for p, (i, j) in enumerate(pairs):
        want = blk(u[i] * u[j]) - blk(u[i]) * blk(u[j])
        assert np.max(np.abs(tau[p] - want)) < 1e-13


def _np_truncate(f):
    """numpy's 2/3 truncation of real fields [..., m, m, m] (keep 3|k_i| < m)."""
    m = f.shape[-1]
    F = np.fft.rfftn(f, axes=(-3, -2, -1))
    a = np.arange(m)
    k = np.where(2 * a < m, a, a - m)
    KX, KY, KZ = np.meshgrid(k, k, np.arange(m // 2 + 1), indexing="ij")
    keep = (3 * np.abs(KX) < m) & (3 * np.abs(KY) < m) & (3 * KZ < m)
    return np.fft.irfftn(F * keep, s=(m, m, m), axes=(-3, -2, -1))


_PAIRS = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]


def test_les_stress_against_numpy_from_a_fine_field(oracle_mod):
    # tau_les = T[<u_i u_j> - (T ubar)_i (T ubar)_j] with the block means and
    # the truncation both done by numpy on a seeded fine field
    n, f = 32, 4
    m = n // f
    u = np.stack([synth.uniform_pm1(3, c, (n, n, n)).astype(np.float64) for c in range(3)])
    ubar, tau = oracle_mod.box_filter(u, f)
    got = oracle_mod.les_stress(ubar, tau)
    blocks = lambda a: a.reshape(m, f, m, f, m, f).mean(axis=(1, 3, 5))
    ub = np.stack([blocks(u[c]) for c in range(3)])
    ut = _np_truncate(ub)
    want = np.stack([_np_truncate(blocks(u[i] * u[j]) - ut[i] * ut[j]) for (i, j) in _PAIRS])
    assert np.max(np.abs(got - want)) < 1e-13


def test_les_stress_of_a_band_limited_filtered_field_is_the_truncated_stress(oracle_mod):
    # when ubar already lies in the kept set, T ubar = ubar and tau_les = T tau
    m = 12
    g = 2 * np.pi * np.arange(m) / m
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    ubar = np.stack([np.sin(X + 2 * Y), np.cos(3 * Z) * 0.5, np.sin(Y - Z)])
    tau = np.stack([synth.uniform_pm1(5, p, (m, m, m)).astype(np.float64) for p in range(6)])
    got = oracle_mod.les_stress(ubar, tau)
    assert np.max(np.abs(got - _np_truncate(tau))) < 1e-13
