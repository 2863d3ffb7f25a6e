"""GPU parity of the fused Navier-Stokes path (tarang_ns_rhs, tarang_ns_step,
tarang_diag) against the FP64 oracle, through the C ABI.

Inputs are the oracle's initial fields rounded to complex64, fed to both sides.
Tolerances follow from FP32 arithmetic (u = 2^-24): each of the nine 3D
transforms of a right-hand side contributes ~u log2(N^3) relative error, the
products and projection a few u more, so the right-hand side is held to
relative L2 <= 1e-5; states after a few steps inherit that error only through
the increments dt*N, and the per-shell spectrum to relative 1e-4 on
shells holding >= 1e-8 of the peak shell energy.
"""
import json
import os

import numpy as np
import pytest

import synth
from gpu_helpers import empty_c64, from_dev_c64, rel_l2, stream, sync, to_dev_c64

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def fk():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_07801_gb300 import build as b

    b.build()
    import paper_1805_07801_gb300 as m

    return m


class Plan:
    def __init__(self, fk, n):
        self.fk = fk
        self.h = fk.fftk_plan_create(n, n, n)

    def __enter__(self):
        return self.h

    def __exit__(self, *a):
        self.fk.fftk_plan_destroy(self.h)


def _kvec(n):
    a = np.arange(n)
    kx = np.where(2 * a < n, a, a - n)
    return np.meshgrid(kx, kx, np.arange(n // 2 + 1), indexing="ij")


def _kept(n):
    KX, KY, KZ = _kvec(n)
    return (3 * np.abs(KX) < n) & (3 * np.abs(KY) < n) & (3 * np.abs(KZ) < n)


def random_ic(oracle_mod, n, seed=0, k0=2.0, E0=0.5):
    u = oracle_mod.ic_random(synth.normal_fields(seed, 3, (n, n, n)), k0=k0, E0=E0)
    return u.astype(np.complex64)


def gpu_rhs(fk, plan, u64, nu=0.0, feps=0.0, k2=(1, 4)):
    ud = to_dev_c64(u64)
    nd = empty_c64(u64.shape)
    fk.tarang_ns_rhs(plan, ud.data_ptr(), nd.data_ptr(), fk.make_params(nu, 0.0, feps, k2), stream())
    sync()
    return from_dev_c64(nd)


def gpu_steps(fk, plan, u64, nu, dt, nsteps, feps=0.0, k2=(1, 4)):
    ud = to_dev_c64(u64)
    d = fk.tarang_ns_step(plan, ud.data_ptr(), fk.make_params(nu, dt, feps, k2), nsteps, True, stream())
    return from_dev_c64(ud), d


def shells_ok(EKg, EKo, rel=1e-4, floor=1e-8):
    EKg = np.asarray(EKg)
    EKo = np.asarray(EKo)
    m = min(len(EKg), len(EKo))
    EKg, EKo = EKg[:m], EKo[:m]
    res = EKo >= floor * EKo.max()
    relerr = np.abs(EKg[res] - EKo[res]) / EKo[res]
    abserr = np.abs(EKg[~res] - EKo[~res])
    return relerr.max(), (abserr.max() if abserr.size else 0.0), int(np.nonzero(res)[0].max())


@pytest.mark.parametrize("n", [8, 16, 32, 64])
def test_rhs_matches_oracle(fk, oracle_mod, n):
    u = random_ic(oracle_mod, n, seed=n, k0=min(4.0, n / 8))
    with Plan(fk, n) as plan:
        Ng = gpu_rhs(fk, plan, u)
    No = oracle_mod.ns_rhs(u.astype(np.complex128))
    assert rel_l2(Ng, No) < 1e-5
    assert np.all(Ng[:, ~_kept(n)] == 0)


def test_rhs_taylor_green_is_zero(fk, oracle_mod):
    n = 32
    u = oracle_mod.ic_taylor_green(n).astype(np.complex64)
    with Plan(fk, n) as plan:
        Ng = gpu_rhs(fk, plan, u)
    assert np.max(np.abs(Ng)) < 1e-7


def test_rhs_shear_pair_closed_form(fk, oracle_mod):
    n = 16
    g = 2 * np.pi * np.arange(n) / n
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    u = oracle_mod.rfft3(np.stack([np.sin(Y), 0 * X, np.sin(X)])).astype(np.complex64)
    want = np.fft.rfftn(np.stack([0 * X, 0 * X, -np.cos(X) * np.sin(Y)]), axes=(1, 2, 3)) / n**3
    with Plan(fk, n) as plan:
        Ng = gpu_rhs(fk, plan, u)
    assert np.max(np.abs(Ng - want)) < 1e-7


def test_rhs_invariants_and_forcing(fk, oracle_mod):
    n = 32
    u = random_ic(oracle_mod, n, seed=5, k0=3.0)
    with Plan(fk, n) as plan:
        N0 = gpu_rhs(fk, plan, u)
        Nf = gpu_rhs(fk, plan, u, feps=0.1, k2=(1, 4))
    uw = u.astype(np.complex128)
    scale = np.sqrt(np.sum(np.abs(N0) ** 2) * np.sum(np.abs(uw) ** 2))
    assert abs(oracle_mod.transfer(uw, N0)) < 1e-6 * scale
    assert abs(oracle_mod.transfer(uw, Nf) - 0.1) < 1e-5
    KX, KY, KZ = _kvec(n)
    div = KX * N0[0] + KY * N0[1] + KZ * N0[2]
    assert np.max(np.abs(div)) < 1e-6 * np.max(np.abs(N0)) * n
    No = oracle_mod.ns_rhs(uw, force_eps=0.1, force_k2=(1, 4))
    assert rel_l2(Nf, No) < 1e-5


def test_taylor_green_decay_config_small(fk, oracle_mod):
    # 64^3 extruded Taylor-Green, nu = 0.01, dt = 1e-3, 20 steps:
    # exact decay E(t) = 1/4 exp(-4 nu t) and the oracle's state
    n, nu, dt, steps = 64, 0.01, 1e-3, 20
    u0 = oracle_mod.ic_taylor_green(n).astype(np.complex64)
    with Plan(fk, n) as plan:
        ug, (E, eps, EK) = gpu_steps(fk, plan, u0, nu, dt, steps)
    t = steps * dt
    # one FP32 rounding of u * E per step (0.5 ulp, relative 2^-24 worst case),
    # twice that in the energy: |dE/E| <= 2 * 20 * 2^-24 = 2.4e-6
    assert abs(E - 0.25 * np.exp(-4 * nu * t)) < 2.4e-6 * 0.25
    assert abs(eps - 2 * nu * 2 * 0.25 * np.exp(-4 * nu * t)) < 1e-5 * eps
    uo = oracle_mod.ns_step(u0.astype(np.complex128), nu, dt, steps)
    assert rel_l2(ug, uo) < 1.2e-6


def test_taylor_green_long_run_decay_is_unbiased(fk, oracle_mod):
    # 4000 steps: the integrating factor is applied as an FP64-accurate FP32
    # pair, so the per-step roundings are unbiased (random walk ~ sqrt(4000)
    # * 2^-25 = 1.9e-6) instead of accumulating a fixed factor error (up to
    # 4000 * 2^-25 = 1.2e-4 for a factor rounded once to FP32).
    n, nu, dt, steps = 16, 0.01, 1e-3, 4000
    u0 = oracle_mod.ic_taylor_green(n).astype(np.complex64)
    with Plan(fk, n) as plan:
        _, (E, _, _) = gpu_steps(fk, plan, u0, nu, dt, steps)
    exact = 0.25 * np.exp(-4 * nu * steps * dt)
    assert abs(E - exact) < 2e-5 * exact


def test_random_decay_matches_oracle(fk, oracle_mod):
    n, nu, dt, steps = 64, 1e-3, 5e-4, 10
    u0 = random_ic(oracle_mod, n, seed=0, k0=4.0)
    with Plan(fk, n) as plan:
        ug, (E, eps, EK) = gpu_steps(fk, plan, u0, nu, dt, steps)
    uo = oracle_mod.ns_step(u0.astype(np.complex128), nu, dt, steps)
    Eo, epso, EKo = oracle_mod.diag(uo, nu)
    assert rel_l2(ug, uo) < 1e-5
    assert abs(E - Eo) < 1e-6 * Eo
    assert abs(eps - epso) < 1e-5 * epso
    r, a, kres = shells_ok(EK, EKo)
    assert r < 1e-4 and a < 1e-10 * Eo


def test_forced_steps_match_oracle(fk, oracle_mod):
    n, nu, dt, steps = 32, 4e-4, 2.5e-4, 10
    u0 = random_ic(oracle_mod, n, seed=1, k0=2.0)
    with Plan(fk, n) as plan:
        ug, (E, eps, EK) = gpu_steps(fk, plan, u0, nu, dt, steps, feps=0.1, k2=(1, 4))
    uo = oracle_mod.ns_step(u0.astype(np.complex128), nu, dt, steps, force_eps=0.1, force_k2=(1, 4))
    Eo, epso, _ = oracle_mod.diag(uo, nu)
    assert rel_l2(ug, uo) < 1e-5
    assert abs(E - Eo) < 1e-6 * Eo


def test_diag_matches_oracle_and_is_bitwise_reproducible(fk, oracle_mod):
    n = 64
    u = random_ic(oracle_mod, n, seed=7, k0=4.0)
    with Plan(fk, n) as plan:
        ud = to_dev_c64(u)
        d1 = fk.tarang_diag(plan, ud.data_ptr(), 1e-3, stream())
        d2 = fk.tarang_diag(plan, ud.data_ptr(), 1e-3, stream())
        assert len(d1[2]) == fk.tarang_diag_kmax(plan) + 1
    assert d1 == d2
    Eo, epso, EKo = oracle_mod.diag(u.astype(np.complex128), 1e-3)
    assert abs(d1[0] - Eo) < 1e-13
    assert abs(d1[1] - epso) < 1e-13 * max(1.0, epso) * 10
    assert np.max(np.abs(np.asarray(d1[2]) - EKo[: len(d1[2])])) < 1e-14


def test_step_launch_count_and_state_of_dropped_modes(fk, oracle_mod):
    n = 32
    u0 = random_ic(oracle_mod, n, seed=3, k0=3.0)
    with Plan(fk, n) as plan:
        ud = to_dev_c64(u0)
        c0 = fk.fftk_launch_count(plan)
        fk.tarang_ns_step(plan, ud.data_ptr(), fk.make_params(1e-3, 1e-3), 2, False, stream())
        sync()
        assert fk.fftk_launch_count(plan) - c0 == 2 * 2 * 5
        u1 = from_dev_c64(ud)
    assert np.all(u1[:, ~_kept(n)] == 0)


def test_argument_errors(fk):
    with Plan(fk, 32) as plan:
        import torch

        buf = torch.zeros(3 * 32 * 32 * 17 * 2, dtype=torch.float32, device="cuda:0")
        p = buf.data_ptr()
        for prm in [fk.make_params(-1.0, 1e-3), fk.make_params(1e-3, 0.0), fk.make_params(1e-3, 1e-3, 0.1, (1, 200))]:
            with pytest.raises(fk.FFTKError) as e:
                fk.tarang_ns_step(plan, p, prm, 1, False, stream())
            assert e.value.status == fk.FFTK_ERR_INVALID_ARG
        with pytest.raises(fk.FFTKError) as e:
            fk.tarang_ns_rhs(plan, p, p, fk.make_params(1e-3), stream())
        assert e.value.status == fk.FFTK_ERR_INVALID_ARG
    plan = fk.fftk_plan_create(32, 32, 16)
    try:
        with pytest.raises(fk.FFTKError) as e:
            fk.tarang_ns_step(plan, p, fk.make_params(1e-3, 1e-3), 1, False, stream())
        assert e.value.status == fk.FFTK_ERR_UNSUPPORTED_SIZE
    finally:
        fk.fftk_plan_destroy(plan)


def _golden_decay(fk, oracle_mod, n):
    path = os.path.join(GOLDEN, f"ns{n}_decay_100steps.json")
    if not os.path.exists(path):
        pytest.skip(f"{path} not generated")
    gold = json.load(open(path))
    cfg = gold["config"]
    u0 = random_ic(oracle_mod, n, seed=cfg["seed"], k0=cfg["k0"], E0=cfg["E0"])
    csum = float(np.sum(np.abs(u0.astype(np.complex128)) ** 2 * np.arange(1, u0.shape[-1] + 1)))
    assert abs(csum - gold["ic_checksum"]) <= 1e-12 * abs(gold["ic_checksum"])
    with Plan(fk, n) as plan:
        _, (E, eps, EK) = gpu_steps(fk, plan, u0, cfg["nu"], cfg["dt"], cfg["steps"])
    fin = gold["final"]
    assert abs(E - fin["E"]) < 1e-5 * fin["E"]
    assert abs(eps - fin["eps"]) < 1e-4 * fin["eps"]
    r, a, kres = shells_ok(EK, fin["EK"])
    assert r < 1e-4, (r, kres)
    assert a < 1e-10 * fin["E"]


def test_decay_64_100_steps_vs_stored_oracle(fk, oracle_mod):
    _golden_decay(fk, oracle_mod, 64)


def test_decay_512_100_steps_vs_stored_oracle(fk, oracle_mod):
    """The 512^3 decaying-turbulence workload: per-shell spectrum after 100
    steps vs the oracle's stored run (tests/golden/make_ns512_golden.py)."""
    _golden_decay(fk, oracle_mod, 512)


def test_diag_after_smaller_plan(fk, oracle_mod):
    """A smaller plan's solver state must not shrink the reduction kernel's
    shared-memory limit under a larger plan (the limit is per kernel)."""
    u = random_ic(oracle_mod, 64, seed=3)
    with Plan(fk, 64) as big:
        ud = to_dev_c64(u)
        first = fk.tarang_diag(big, ud.data_ptr(), 1e-3, stream())
        with Plan(fk, 16) as small:
            us = to_dev_c64(random_ic(oracle_mod, 16, seed=4))
            fk.tarang_diag(small, us.data_ptr(), 1e-3, stream())
            again = fk.tarang_diag(big, ud.data_ptr(), 1e-3, stream())
    assert first[0] == again[0] and first[2] == again[2]
