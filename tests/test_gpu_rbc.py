"""GPU parity of the Rayleigh-Benard solver (tarang_rbc_rhs, tarang_rbc_step;
Sec. 2.2, Eqs. (12)-(13), FFF basis) against the FP64 oracle, through the C
ABI.  The right-hand side goes through 13 FP32 transforms and pointwise
products: relative L2 1e-5, as for the Navier-Stokes right-hand side; states
after a few steps inherit it through dt N.
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


def _state(oracle_mod, n, seed, k0=2.0):
    u = oracle_mod.ic_random(synth.normal_fields(seed, 3, (n, n, n)), k0=k0, E0=0.5)
    th = np.fft.rfftn(synth.normal(seed + 1, 0, (n, n, n)).astype(np.float64)) / n**3
    KX, KY, KZ = _kvec(n)
    keep = (3 * np.abs(KX) < n) & (3 * np.abs(KY) < n) & (3 * np.abs(KZ) < n)
    th = np.where(keep, th * np.exp(-(KX**2 + KY**2 + KZ**2) / (2 * k0 * k0)), 0.0)
    th[0, 0, 0] = 0.0
    th *= np.sqrt(0.1 / (0.5 * np.sum(np.where(KZ == 0, 1.0, 2.0) * np.abs(th) ** 2)))  # 1/2 <theta^2> = 0.1
    return np.concatenate([u, th[None]], axis=0).astype(np.complex64)


@pytest.mark.parametrize("n", [16, 32, 64])
def test_rbc_rhs_matches_oracle(fk, oracle_mod, n):
    s = _state(oracle_mod, n, 40 + n)
    plan = fk.fftk_plan_create(n, n, n)
    try:
        sd = to_dev_c64(s)
        od = to_dev_c64(np.zeros_like(s))
        fk.tarang_rbc_rhs(plan, sd.data_ptr(), od.data_ptr(), stream())
        sync()
        got = from_dev_c64(od)
    finally:
        fk.fftk_plan_destroy(plan)
    want = oracle_mod.rbc_rhs(s.astype(np.complex128))
    assert rel_l2(got[:3], want[:3]) < 1e-5
    assert rel_l2(got[3], want[3]) < 1e-5
    KX, KY, KZ = _kvec(n)
    keep = (3 * np.abs(KX) < n) & (3 * np.abs(KY) < n) & (3 * np.abs(KZ) < n)
    assert np.all(got[:, ~keep] == 0)


@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("n", [32, 64])
def test_rbc_steps_match_oracle(fk, oracle_mod, n, scheme):
    Ra, Pr, dt, steps = 1e5, 1.0, 2e-3, 8
    s = _state(oracle_mod, n, 50 + n)
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
    # u perpendicular to k: no nonlinear interaction; amplitude and temperature
    # follow the 2x2 linear system exactly (growth rate from its eigenvalues)
    n, kx, kz, A, B = 32, 2, 1, 0.3, -0.7
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
        real = np.stack([a * e[0] * c, a * e[1] * c, a * e[2] * c, b * c])
        return np.fft.rfftn(real, axes=(1, 2, 3)) / n**3

    plan = fk.fftk_plan_create(n, n, n)
    try:
        sd = to_dev_c64(wave(A, B))
        fk.tarang_rbc_step(plan, sd.data_ptr(), Ra, Pr, dt, steps, fk.TARANG_RK4, stream())
        sync()
        got = from_dev_c64(sd)
    finally:
        fk.fftk_plan_destroy(plan)
    want = wave(A1, B1)
    # 300 steps of FP32 rounding of a single mode: ~300 * 2^-24 relative
    assert np.max(np.abs(got - want)) < 3e-5 * np.max(np.abs(want))
    assert abs(B1) > 1.5 * abs(B)


def test_rbc_full_size_energy_exchange(fk):
    # 512^3, nearly inviscid (Ra = 1e12, Pr = 1): advection conserves 1/2|u|^2
    # and 1/2 theta^2 separately and buoyancy moves the same amount <u_z theta>
    # into both, so E_u - E_theta stays constant while E_u changes
    import torch

    n, Ra, Pr, dt, steps = 512, 1e12, 1.0, 1e-3, 10
    dev = torch.device("cuda:0")
    st = stream()
    plan = fk.fftk_plan_create(n, n, n)
    try:
        nr = torch.empty((3, n, n, n), dtype=torch.float32, device=dev)
        for f in range(3):
            fk.fftk_fill_normal(nr[f].data_ptr(), n**3, 7, f, st)
        s = torch.empty((4, n, n, n // 2 + 1, 2), dtype=torch.float32, device=dev)
        fk.tarang_ic_random(plan, nr.data_ptr(), s.data_ptr(), 4.0, 0.5, st)
        s[3].copy_(s[2])  # theta = u_z: a warm rising plume everywhere, <u_z theta> > 0
        del nr
        w = torch.full((n // 2 + 1,), 2.0, dtype=torch.float64, device=dev)
        w[0] = 1.0
        w[n // 2] = 1.0

        def energies():
            Eu = fk.tarang_diag(plan, s.data_ptr(), 0.0, st)[0]
            t = s[3].double()
            Et = 0.5 * float(((t[..., 0] ** 2 + t[..., 1] ** 2) * w).sum())
            return Eu, Et

        Eu0, Et0 = energies()
        fk.tarang_rbc_step(plan, s.data_ptr(), Ra, Pr, dt, steps, fk.TARANG_RK4, st)
        Eu1, Et1 = energies()
    finally:
        fk.fftk_plan_destroy(plan)
    assert abs(Eu1 - Eu0) > 1e-4
    assert abs((Eu1 - Et1) - (Eu0 - Et0)) < 1e-3 * abs(Eu1 - Eu0)


def test_rbc_argument_errors(fk):
    import torch

    plan = fk.fftk_plan_create(16, 16, 16)
    try:
        s = torch.zeros((4, 16, 16, 9, 2), device="cuda:0")
        for Ra, Pr, dt, sch in ((0.0, 1.0, 1e-3, 1), (1e4, -1.0, 1e-3, 1), (1e4, 1.0, 0.0, 1), (1e4, 1.0, 1e-3, 5)):
            with pytest.raises(fk.FFTKError):
                fk.tarang_rbc_step(plan, s.data_ptr(), Ra, Pr, dt, 1, sch, stream())
        with pytest.raises(fk.FFTKError):
            fk.tarang_rbc_rhs(plan, s.data_ptr(), s.data_ptr(), stream())
    finally:
        fk.fftk_plan_destroy(plan)
