"""Pins for the oracle's convection between free-slip, isothermal plates (the
SFF basis; Sec. 2.2, Eqs. (12)-(14)): wall-normal axis x on [0, pi] with
gravity along it, u_x and theta in the sine basis, u_y and u_z in the
cosine basis, y and z periodic.

The classic convection roll at vanishing amplitude follows the exact 2x2
linear system; the projected term is divergence-free in the mixed basis;
advection conserves 1/2 |u|^2 and 1/2 theta^2 (checked on the grid, where
band-limited products are exact); RK4 is fourth order.
"""
import numpy as np
import pytest


def _grids(n):
    x = (np.arange(n) + 0.5) * np.pi / n
    y = 2 * np.pi * np.arange(n) / n
    return np.meshgrid(x, y, y, indexing="ij")


def _to_state(oracle_mod, ux, uy, uz, th):
    return np.stack([oracle_mod.transform3(ux, "SFF"), oracle_mod.transform3(uy, "CFF"),
                     oracle_mod.transform3(uz, "CFF"), oracle_mod.transform3(th, "SFF")])


def _to_real(oracle_mod, s, n):
    return (oracle_mod.itransform3(s[0], n, "SFF"), oracle_mod.itransform3(s[1], n, "CFF"),
            oracle_mod.itransform3(s[2], n, "CFF"), oracle_mod.itransform3(s[3], n, "SFF"))


def _roll(oracle_mod, n, kx, ky, A, B):
    X, Y, Z = _grids(n)
    ux = A * np.sin(kx * X) * np.cos(ky * Y)
    uy = -A * (kx / ky) * np.cos(kx * X) * np.sin(ky * Y)
    th = B * np.sin(kx * X) * np.cos(ky * Y)
    return _to_state(oracle_mod, ux, uy, 0 * X, th)


def _random_solenoidal(oracle_mod, n, seed):
    # u = curl(psi1 z) + curl(psi2 y), psi sine in x: solenoidal, u_x = 0 on the plates
    rng = np.random.default_rng(seed)
    X, Y, Z = _grids(n)
    ux = np.zeros_like(X)
    uy = np.zeros_like(X)
    uz = np.zeros_like(X)
    th = np.zeros_like(X)
    for _ in range(6):
        kx, ky, kz = rng.integers(1, 4), rng.integers(-3, 4), rng.integers(0, 4)
        a1, a2, a3, ph = rng.standard_normal(4)
        arg = ky * Y + kz * Z + ph
        # psi1 = a1 sin(kx x) cos(arg):  u_x += d_y psi1, u_y -= d_x psi1
        ux += -a1 * ky * np.sin(kx * X) * np.sin(arg)
        uy += -a1 * kx * np.cos(kx * X) * np.cos(arg)
        # psi2 = a2 sin(kx x) cos(arg):  u_x -= d_z psi2, u_z += d_x psi2
        ux += a2 * kz * np.sin(kx * X) * np.sin(arg)
        uz += a2 * kx * np.cos(kx * X) * np.cos(arg)
        th += a3 * np.sin(kx * X) * np.cos(arg)
    return _to_state(oracle_mod, ux, uy, uz, th)


def _kx_ky_kz(n):
    a = np.arange(n)
    ky = np.where(2 * a < n, a, a - n)
    return np.meshgrid(a, ky, np.arange(n // 2 + 1), indexing="ij")


def test_roll_follows_the_exact_linear_solution(oracle_mod):
    n, kx, ky = 16, 1, 2
    Ra, Pr, dt, steps = 2e3, 1.0, 2e-2, 100
    nu, kappa = np.sqrt(Pr / Ra), 1 / np.sqrt(Ra * Pr)
    k2 = kx * kx + ky * ky
    Mx = np.array([[-nu * k2, ky * ky / k2], [1.0, -kappa * k2]])
    lam, V = np.linalg.eig(Mx)
    A0, B0 = 1e-10, 2e-10
    A1, B1 = np.real(V @ (np.exp(lam * dt * steps) * np.linalg.solve(V, np.array([A0, B0]))))
    s = oracle_mod.rbc_sff_step(_roll(oracle_mod, n, kx, ky, A0, B0), Ra, Pr, dt, steps, 1)
    want = _roll(oracle_mod, n, kx, ky, A1, B1)
    assert np.max(np.abs(s - want)) < 1e-8 * np.max(np.abs(want))
    assert abs(B1) > 3 * abs(B0)  # above onset: the roll grows


def test_projected_term_is_divergence_free(oracle_mod):
    n = 16
    s = _random_solenoidal(oracle_mod, n, 1)
    N = oracle_mod.rbc_sff_rhs(s)
    KX, KY, KZ = _kx_ky_kz(n)
    nxs = np.zeros_like(N[0])
    nxs[1:] = N[0][:-1]  # the sine coefficient of k_x = a sits at index a - 1
    div = KX * nxs + 1j * KY * N[1] + 1j * KZ * N[2]
    assert np.max(np.abs(N[:3])) > 1e-2
    assert np.max(np.abs(div)) < 1e-13 * np.max(np.abs(N[:3])) * n


def test_advection_conserves_energies_on_the_grid(oracle_mod):
    n = 16
    s = _random_solenoidal(oracle_mod, n, 2)
    # u alone: the velocity term conserves 1/2 |u|^2
    s0 = s.copy()
    s0[3] = 0
    N = oracle_mod.rbc_sff_rhs(s0)
    u = _to_real(oracle_mod, s0, n)
    Nr = _to_real(oracle_mod, N, n)
    pw = np.mean(u[0] * Nr[0] + u[1] * Nr[1] + u[2] * Nr[2])
    scale = np.mean(np.abs(u[0] * Nr[0]) + np.abs(u[1] * Nr[1]) + np.abs(u[2] * Nr[2]))
    assert scale > 1e-3 and abs(pw) < 1e-13 * scale
    # temperature advection conserves 1/2 theta^2 (the u_x source aside)
    N = oracle_mod.rbc_sff_rhs(s)
    r = _to_real(oracle_mod, s, n)
    Nr = _to_real(oracle_mod, N, n)
    adv = Nr[3] - r[0]
    pt = np.mean(r[3] * adv)
    scale_t = np.mean(np.abs(r[3] * adv))
    assert scale_t > 1e-3 and abs(pt) < 1e-13 * scale_t


def test_buoyancy_alone(oracle_mod):
    # u = 0: N_u = P[theta x], N_theta = 0; for theta = sin(kx x) cos(ky y),
    # P[theta x]_x = theta ky^2 / k^2
    n, kx, ky = 16, 2, 3
    X, Y, Z = _grids(n)
    th = np.sin(kx * X) * np.cos(ky * Y)
    s = _to_state(oracle_mod, 0 * X, 0 * X, 0 * X, th)
    N = oracle_mod.rbc_sff_rhs(s)
    assert np.max(np.abs(N[3])) < 1e-15
    assert np.max(np.abs(N[0] - s[3] * ky * ky / (kx * kx + ky * ky))) < 1e-15


def test_sff_rk4_is_fourth_order(oracle_mod):
    n, Ra, Pr, T = 16, 1e4, 1.0, 0.2
    s0 = _random_solenoidal(oracle_mod, n, 3) * 0.2
    ref = oracle_mod.rbc_sff_step(s0, Ra, Pr, T / 64, 64, 1)
    e = [np.linalg.norm(oracle_mod.rbc_sff_step(s0, Ra, Pr, T / m, m, 1) - ref) for m in (4, 8)]
    assert 13.0 < e[0] / e[1] < 19.0, e


class _Term:
    """amp * fx(kx x) * fa(ky y + kz z + ph), fx, fa in {sin, cos}, with exact derivatives."""

    def __init__(self, amp, fx, kx, fa, ky, kz, ph):
        self.amp, self.fx, self.kx, self.fa, self.ky, self.kz, self.ph = amp, fx, kx, fa, ky, kz, ph

    def value(self, X, Y, Z):
        gx = np.sin if self.fx == "s" else np.cos
        ga = np.sin if self.fa == "s" else np.cos
        return self.amp * gx(self.kx * X) * ga(self.ky * Y + self.kz * Z + self.ph)

    def d(self, axis):
        t = _Term(self.amp, self.fx, self.kx, self.fa, self.ky, self.kz, self.ph)
        if axis == 0:
            t.amp *= self.kx if self.fx == "s" else -self.kx
            t.fx = "c" if self.fx == "s" else "s"
        else:
            k = self.ky if axis == 1 else self.kz
            t.amp *= k if self.fa == "s" else -k
            t.fa = "c" if self.fa == "s" else "s"
        return t


def _field_terms(seed):
    # u = curl(psi1 z) + curl(psi2 y) with psi = a sin(kx x) cos(arg): terms per
    # component; wavenumbers low enough that products stay inside the kept set
    # at n = 16 (|k_y|, k_z <= 4 < 16/3)
    rng = np.random.default_rng(seed)
    comps = [[], [], []]
    th = []
    for _ in range(6):
        kx, ky, kz = int(rng.integers(1, 4)), int(rng.integers(-2, 3)), int(rng.integers(0, 3))
        a1, a2, a3, ph = rng.standard_normal(4)
        p1 = _Term(a1, "s", kx, "c", ky, kz, ph)
        p2 = _Term(a2, "s", kx, "c", ky, kz, ph)
        comps[0] += [p1.d(1)]
        comps[1] += [_neg(p1.d(0))]
        comps[0] += [_neg(p2.d(2))]
        comps[2] += [p2.d(0)]
        th += [_Term(a3, "s", kx, "c", ky, kz, ph)]
    return comps, th


def _neg(t):
    t.amp = -t.amp
    return t


def _eval(terms, G):
    return sum(t.value(*G) for t in terms)


def test_velocity_term_against_advective_form(oracle_mod):
    # <v, N_u> = <v, -(u.grad)u + theta x> for solenoidal v with v_x = 0 on the
    # plates (the pressure gradient is orthogonal to them); every product is
    # band-limited, so grid means are exact
    n = 16
    G = _grids(n)
    comps, th = _field_terms(4)
    u = [_eval(c, G) for c in comps]
    grad = [[_eval([t.d(j) for t in comps[i]], G) for j in range(3)] for i in range(3)]
    t = _eval(th, G)
    adv = [-(u[0] * grad[i][0] + u[1] * grad[i][1] + u[2] * grad[i][2]) for i in range(3)]
    adv[0] = adv[0] + t
    s = _to_state(oracle_mod, u[0], u[1], u[2], t)
    Nr = _to_real(oracle_mod, oracle_mod.rbc_sff_rhs(s), n)
    for seed in (5, 6, 7):
        vc, _ = _field_terms(seed)
        v = [_eval(c, G) for c in vc]
        lhs = np.mean(v[0] * Nr[0] + v[1] * Nr[1] + v[2] * Nr[2])
        rhs = np.mean(v[0] * adv[0] + v[1] * adv[1] + v[2] * adv[2])
        assert abs(rhs) > 1e-2
        assert abs(lhs - rhs) < 1e-12 * np.mean(np.abs(v[0] * adv[0]) + np.abs(v[1] * adv[1]) + np.abs(v[2] * adv[2]))
    # the temperature term is -u.grad theta + u_x exactly (no projection)
    tg = [_eval([tt.d(j) for tt in th], G) for j in range(3)]
    want = -(u[0] * tg[0] + u[1] * tg[1] + u[2] * tg[2]) + u[0]
    assert np.max(np.abs(Nr[3] - want)) < 1e-12 * np.max(np.abs(want))
