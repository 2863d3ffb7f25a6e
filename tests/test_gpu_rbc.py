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


# ------------------------------------------------- free-slip plates (SFF) --
def _sff_state(oracle_mod, n, seed, k0=3.0):
    # smooth random fields: normal noise -> mixed-basis transform -> Gaussian
    # taper -> truncation 3 k_x < 2n, 3|k_y| < n, 3 k_z < n
    a = np.arange(n)
    ky = np.where(2 * a < n, a, a - n)
    KA, KY, KZ = np.meshgrid(a, ky, np.arange(n // 2 + 1), indexing="ij")
    out = []
    for f, basis in enumerate(("SFF", "CFF", "CFF", "SFF")):
        F = oracle_mod.transform3(synth.normal(seed, f, (n, n, n)).astype(np.float64), basis)
        kx = KA + 1 if basis[0] == "S" else KA
        keep = (3 * kx < 2 * n) & (3 * np.abs(KY) < n) & (3 * KZ < n)
        out.append(np.where(keep, F * np.exp(-(kx**2 + KY**2 + KZ**2) / (2 * k0 * k0)) * n, 0.0))
    return np.stack(out).astype(np.complex64)


@pytest.mark.parametrize("n", [16, 32, 64])
def test_sff_rhs_matches_oracle(fk, oracle_mod, n):
    s = _sff_state(oracle_mod, n, 60 + n)
    plan = fk.fftk_plan_create(n, n, n)
    try:
        sd = to_dev_c64(s)
        od = to_dev_c64(np.zeros_like(s))
        fk.tarang_rbc_rhs(plan, sd.data_ptr(), od.data_ptr(), stream(), basis=fk.TARANG_RBC_SFF)
        sync()
        got = from_dev_c64(od)
    finally:
        fk.fftk_plan_destroy(plan)
    want = oracle_mod.rbc_sff_rhs(s.astype(np.complex128))
    assert np.max(np.abs(want[:3])) > 1e-3 and np.max(np.abs(want[3])) > 1e-3
    assert rel_l2(got[:3], want[:3]) < 1e-5
    assert rel_l2(got[3], want[3]) < 1e-5


@pytest.mark.parametrize("scheme", [0, 1])
def test_sff_steps_match_oracle(fk, oracle_mod, scheme):
    n, Ra, Pr, dt, steps = 32, 1e5, 1.0, 2e-3, 8
    s = _sff_state(oracle_mod, n, 70 + scheme)
    plan = fk.fftk_plan_create(n, n, n)
    try:
        sd = to_dev_c64(s)
        fk.tarang_rbc_step(plan, sd.data_ptr(), Ra, Pr, dt, steps, scheme, stream(), basis=fk.TARANG_RBC_SFF)
        sync()
        got = from_dev_c64(sd)
    finally:
        fk.fftk_plan_destroy(plan)
    want = oracle_mod.rbc_sff_step(s.astype(np.complex128), Ra, Pr, dt, steps, scheme)
    assert rel_l2(got[:3], want[:3]) < 1e-5
    assert rel_l2(got[3], want[3]) < 1e-5


def test_sff_roll_grows_as_the_exact_solution(fk, oracle_mod):
    # the classic roll u_x = A sin(kx x) cos(ky y), theta = B sin(kx x) cos(ky y)
    # above onset, at an amplitude where advection is negligible
    n, kx, ky = 32, 1, 2
    Ra, Pr, dt, steps = 2e3, 1.0, 2e-2, 100
    nu, kappa = np.sqrt(Pr / Ra), 1 / np.sqrt(Ra * Pr)
    k2 = kx * kx + ky * ky
    lam, V = np.linalg.eig(np.array([[-nu * k2, ky * ky / k2], [1.0, -kappa * k2]]))
    A0, B0 = 1e-6, 2e-6
    A1, B1 = np.real(V @ (np.exp(lam * dt * steps) * np.linalg.solve(V, np.array([A0, B0]))))
    x = (np.arange(n) + 0.5) * np.pi / n
    y = 2 * np.pi * np.arange(n) / n
    X, Y, Z = np.meshgrid(x, y, y, indexing="ij")

    def roll(A, B):
        return np.stack([oracle_mod.transform3(A * np.sin(kx * X) * np.cos(ky * Y), "SFF"),
                         oracle_mod.transform3(-A * (kx / ky) * np.cos(kx * X) * np.sin(ky * Y), "CFF"),
                         oracle_mod.transform3(0 * X, "CFF"),
                         oracle_mod.transform3(B * np.sin(kx * X) * np.cos(ky * Y), "SFF")])

    plan = fk.fftk_plan_create(n, n, n)
    try:
        sd = to_dev_c64(roll(A0, B0))
        fk.tarang_rbc_step(plan, sd.data_ptr(), Ra, Pr, dt, steps, fk.TARANG_RK4, stream(), basis=fk.TARANG_RBC_SFF)
        sync()
        got = from_dev_c64(sd)
    finally:
        fk.fftk_plan_destroy(plan)
    want = roll(A1, B1)
    assert np.max(np.abs(got - want)) < 3e-5 * np.max(np.abs(want))
    assert abs(B1) > 3 * abs(B0)


def test_sff_full_size_energy_exchange(fk, oracle_mod):
    # 512^3 between plates, nearly inviscid: E_u - E_theta is conserved while
    # E_u changes (buoyancy moves <u_x theta> into both).  Energies by the
    # mixed-basis Parseval weights: sine index a < n-1 weight 2, cosine index
    # 0 weight 4, others 2; times the Fourier half-spectrum weights.
    import torch

    n, Ra, Pr, dt, steps = 512, 1e12, 1.0, 1e-3, 10
    dev = torch.device("cuda:0")
    st = stream()
    plan = fk.fftk_plan_create(n, n, n)
    try:
        # a solenoidal u from two smooth stream functions psi1, psi2 (sine along x):
        # u = curl(psi1 z) + curl(psi2 y): u_x = d_y psi1 - d_z psi2 (sine),
        # u_y = -d_x psi1, u_z = d_x psi2 (cosine: d_x of sine index a - 1 is k_x = a)
        s = torch.zeros((4, n, n, n // 2 + 1, 2), dtype=torch.float32, device=dev)
        tmp = torch.empty((n, n, n), dtype=torch.float32, device=dev)
        psi = torch.empty((2, n, n, n // 2 + 1, 2), dtype=torch.float32, device=dev)
        a = torch.arange(n, device=dev, dtype=torch.float32)
        kyv = torch.where(2 * a < n, a, a - n)
        kz = torch.arange(n // 2 + 1, device=dev, dtype=torch.float32)
        kx = a + 1
        k2 = kx[:, None, None] ** 2 + kyv[None, :, None] ** 2 + kz[None, None, :] ** 2
        keep = (3 * kx[:, None, None] < 2 * n) & (3 * kyv.abs()[None, :, None] < n) & (3 * kz[None, None, :] < n)
        for f in range(2):
            fk.fftk_fill_normal(tmp.data_ptr(), n**3, 9, f, st)
            fk.fftk_forward(plan, "SFF", tmp.data_ptr(), psi[f].data_ptr(), 1, st)
            psi[f] *= (torch.exp(-k2 / 32.0) * keep * n).unsqueeze(-1)
        del tmp
        p1 = torch.view_as_complex(psi[0])
        p2 = torch.view_as_complex(psi[1])
        ux = 1j * kyv[None, :, None] * p1 - 1j * kz[None, None, :] * p2
        uy = torch.zeros_like(p1)
        uz = torch.zeros_like(p1)
        uy[1:] = -a[1:, None, None] * p1[:-1]
        uz[1:] = a[1:, None, None] * p2[:-1]
        for f, v in enumerate((ux, uy, uz, ux)):  # theta = u_x: rising where warm
            s[f].copy_(torch.view_as_real(v))
        del psi, p1, p2, ux, uy, uz
        wx_s = torch.full((n,), 2.0, dtype=torch.float64, device=dev)
        wx_c = torch.full((n,), 2.0, dtype=torch.float64, device=dev)
        wx_c[0] = 4.0
        wyz = torch.full((n // 2 + 1,), 2.0, dtype=torch.float64, device=dev)
        wyz[0] = 1.0
        wyz[n // 2] = 1.0

        def energy(f, wx):
            t = s[f].double()
            return 0.5 * float(((t[..., 0] ** 2 + t[..., 1] ** 2) * wx[:, None, None] * wyz[None, None, :]).sum())

        def energies():
            return energy(0, wx_s) + energy(1, wx_c) + energy(2, wx_c), energy(3, wx_s)

        Eu0, Et0 = energies()
        fk.tarang_rbc_step(plan, s.data_ptr(), Ra, Pr, dt, steps, fk.TARANG_RK4, st, basis=fk.TARANG_RBC_SFF)
        Eu1, Et1 = energies()
    finally:
        fk.fftk_plan_destroy(plan)
    assert abs(Eu1 - Eu0) > 1e-3 * Eu0
    assert abs((Eu1 - Et1) - (Eu0 - Et0)) < 1e-3 * abs(Eu1 - Eu0)


def test_rbc_zero_steps_and_zero_state(fk, oracle_mod):
    # nsteps = 0 leaves the state alone; the zero state stays zero (the
    # conduction profile is a steady solution)
    n = 16
    s = _state(oracle_mod, n, 90)
    plan = fk.fftk_plan_create(n, n, n)
    try:
        for basis in (fk.TARANG_RBC_FFF, fk.TARANG_RBC_SFF):
            sd = to_dev_c64(s)
            fk.tarang_rbc_step(plan, sd.data_ptr(), 1e5, 1.0, 1e-3, 0, fk.TARANG_RK4, stream(), basis=basis)
            sync()
            assert np.array_equal(from_dev_c64(sd), s)
            z = to_dev_c64(np.zeros_like(s))
            fk.tarang_rbc_step(plan, z.data_ptr(), 1e5, 1.0, 1e-3, 3, fk.TARANG_RK4, stream(), basis=basis)
            sync()
            assert not np.any(from_dev_c64(z))
    finally:
        fk.fftk_plan_destroy(plan)


@pytest.mark.parametrize("n", [16, 32])
def test_rbc_transfer_matches_oracle(fk, oracle_mod, n):
    # T_u(K) = shell sums of w Re(u* . N_u) - w Re(u_z* theta); T_theta(K) of
    # w Re(theta* N_theta) - w Re(theta* u_z): the oracle's transfer spectrum
    # of the oracle's right-hand side, one component at a time where needed
    s = _state(oracle_mod, n, 120 + n)
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
    Tu, Tt, Pu = np.array(Tu), np.array(Tt), np.array(Pu)
    for got, want in ((Tu, Tu_o), (Tt, Tt_o)):
        scale = np.max(np.abs(want))
        assert scale > 1e-4
        assert np.max(np.abs(got - want)) < 1e-5 * np.sum(np.abs(want))
    # advection only moves energy between shells
    assert abs(tu) < 1e-5 * np.sum(np.abs(Tu)) and abs(tt) < 1e-5 * np.sum(np.abs(Tt))
    assert np.array_equal(Pu, -np.cumsum(Tu))
