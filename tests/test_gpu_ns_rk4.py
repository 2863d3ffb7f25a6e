"""GPU parity of the paper's RK4 time stepper (tarang_params.scheme =
TARANG_RK4; Sec. 2.2, four right-hand sides per step) against the FP64
oracle's RK4, through the C ABI.  Same tolerances as the RK2 tests: the
state after a few steps inherits the right-hand side's FP32 error through
the increments dt N (relative L2 1e-5), the energy to 1e-6.
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


def _ic(oracle_mod, n, seed, k0):
    return oracle_mod.ic_random(synth.normal_fields(seed, 3, (n, n, n)), k0=k0, E0=0.5).astype(np.complex64)


def _steps(fk, n, u0, nu, dt, steps, feps=0.0, k2=(1, 4), split16=False):
    plan = fk.fftk_plan_create(n, n, n, fk.FFTK_R32_SPLIT16 if split16 else fk.FFTK_R32)
    try:
        ud = to_dev_c64(u0)
        d = fk.tarang_ns_step(plan, ud.data_ptr(), fk.make_params(nu, dt, feps, k2, scheme=fk.TARANG_RK4), steps,
                              True, stream())
        return from_dev_c64(ud), d
    finally:
        fk.fftk_plan_destroy(plan)


def test_rk4_taylor_green_exact_decay(fk, oracle_mod):
    n, nu, dt, steps = 32, 0.01, 2e-3, 20
    u0 = oracle_mod.ic_taylor_green(n).astype(np.complex64)
    ug, (E, _, _) = _steps(fk, n, u0, nu, dt, steps)
    t = steps * dt
    # one FP32 rounding per step in the final combination: |dE/E| <= 2 * steps * 2^-24
    assert abs(E - 0.25 * np.exp(-4 * nu * t)) < 2 * steps * 2.0**-24 * 0.25
    assert rel_l2(ug, oracle_mod.ns_step_rk4(u0.astype(np.complex128), nu, dt, steps)) < 2e-6


@pytest.mark.parametrize("n", [32, 64])
def test_rk4_random_decay_matches_oracle(fk, oracle_mod, n):
    nu, dt, steps = 1e-3, 1e-3, 10
    u0 = _ic(oracle_mod, n, seed=20 + n, k0=min(4.0, n / 8))
    ug, (E, eps, EK) = _steps(fk, n, u0, nu, dt, steps)
    uo = oracle_mod.ns_step_rk4(u0.astype(np.complex128), nu, dt, steps)
    Eo, epso, _ = oracle_mod.diag(uo, nu)
    assert rel_l2(ug, uo) < 1e-5
    assert abs(E - Eo) < 1e-6 * Eo
    assert abs(eps - epso) < 1e-5 * epso


def test_rk4_forced_matches_oracle(fk, oracle_mod):
    n, nu, dt, steps = 32, 4e-4, 5e-4, 10
    u0 = _ic(oracle_mod, n, seed=31, k0=2.0)
    ug, (E, _, _) = _steps(fk, n, u0, nu, dt, steps, feps=0.1, k2=(1, 4))
    uo = oracle_mod.ns_step_rk4(u0.astype(np.complex128), nu, dt, steps, force_eps=0.1, force_k2=(1, 4))
    assert rel_l2(ug, uo) < 1e-5
    assert abs(E - oracle_mod.diag(uo, nu)[0]) < 1e-6 * E


def test_rk4_split16_matches_oracle(fk, oracle_mod):
    # the unfused split-precision right-hand side with the same four stages
    n, nu, dt, steps = 32, 1e-3, 1e-3, 5
    u0 = _ic(oracle_mod, n, seed=32, k0=3.0)
    ug, _ = _steps(fk, n, u0, nu, dt, steps, split16=True)
    uo = oracle_mod.ns_step_rk4(u0.astype(np.complex128), nu, dt, steps)
    assert rel_l2(ug, uo) < 2e-5


def test_rk4_launch_count(fk, oracle_mod):
    n = 32
    u0 = _ic(oracle_mod, n, seed=33, k0=3.0)
    plan = fk.fftk_plan_create(n, n, n)
    try:
        ud = to_dev_c64(u0)
        c0 = fk.fftk_launch_count(plan)
        fk.tarang_ns_step(plan, ud.data_ptr(), fk.make_params(1e-3, 1e-3, scheme=fk.TARANG_RK4), 2, False, stream())
        sync()
        assert fk.fftk_launch_count(plan) - c0 == 2 * 4 * 5
        with pytest.raises(fk.FFTKError):
            fk.tarang_ns_step(plan, ud.data_ptr(), fk.make_params(1e-3, 1e-3, scheme=7), 1, False, stream())
    finally:
        fk.fftk_plan_destroy(plan)


def test_rk4_full_size_against_rk2(fk):
    # 512^3 decaying workload, 20 steps: RK2's local error is O((dt k u)^3)
    # per step, below 1e-7 on the shells holding >= 1e-8 of the peak energy,
    # so the two spectra agree there to 1e-3; the RK4 energy drop matches the
    # dissipation integral (trapezoid over the two ends) to 1e-3
    import torch

    n, nu, dt, steps = 512, 1e-3, 5e-4, 20
    dev = torch.device("cuda:0")
    st = stream()
    plan = fk.fftk_plan_create(n, n, n)
    try:
        nr = torch.empty((3, n, n, n), dtype=torch.float32, device=dev)
        for f in range(3):
            fk.fftk_fill_normal(nr[f].data_ptr(), n**3, 0, f, st)
        u = torch.empty((3, n, n, n // 2 + 1, 2), dtype=torch.float32, device=dev)
        fk.tarang_ic_random(plan, nr.data_ptr(), u.data_ptr(), 4.0, 0.5, st)
        del nr
        E0, eps0, _ = fk.tarang_diag(plan, u.data_ptr(), nu, st)
        u2 = u.clone()
        E4, eps4, EK4 = fk.tarang_ns_step(plan, u.data_ptr(), fk.make_params(nu, dt, scheme=fk.TARANG_RK4), steps,
                                         True, st)
        E2, _, EK2 = fk.tarang_ns_step(plan, u2.data_ptr(), fk.make_params(nu, dt), steps, True, st)
    finally:
        fk.fftk_plan_destroy(plan)
    EK4, EK2 = np.array(EK4), np.array(EK2)
    res = EK2 >= 1e-8 * EK2.max()
    assert np.max(np.abs(EK4[res] - EK2[res]) / EK2[res]) < 1e-3
    T = steps * dt
    assert abs((E4 - E0) + 0.5 * (eps0 + eps4) * T) < 1e-3 * abs(E4 - E0)
