"""The Navier-Stokes solver on cubic grids of 3 * 2^m points (the paper's
XC40 sizes, Sec. 6-7): the right-hand side runs through the plan's
transforms (one radix-3 step over power-of-two sub-lines per 1D pass) with
u x omega formed pointwise in real space, then the per-mode update of the
fused path.  Compared with the FP64 oracle on the same complex64 inputs.

Tolerances as for the power-of-two solver: relative L2 <= 1e-5 for a
right-hand side (nine transforms, products, projection); states after a few
steps inherit the error through dt * N.  The 768^3 case uses a band-limited
field (|k_i| <= 85), whose dealiased right-hand side is the same set of
Fourier coefficients on a 768^3 and on a 512^3 grid (products reach
|k_i| <= 170, alias-free on both), so the oracle's 512^3 result fixes every
768^3 coefficient.
"""
import numpy as np
import pytest

import synth
from gpu_helpers import empty_c64, from_dev_c64, rel_l2, stream, sync, to_dev_c64

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


def _rhs(fk, plan, u, feps=0.0):
    ud = to_dev_c64(u)
    nd = empty_c64(u.shape)
    fk.tarang_ns_rhs(plan, ud.data_ptr(), nd.data_ptr(), fk.make_params(0.0, 0.0, feps, (1, 4)), stream())
    fk.fftk_sync(plan, stream())
    return from_dev_c64(nd)


def _kept(n):
    a = np.arange(n)
    k = np.where(2 * a < n, a, a - n)
    KX, KY, KZ = np.meshgrid(k, k, np.arange(n // 2 + 1), indexing="ij")
    return (3 * np.abs(KX) < n) & (3 * np.abs(KY) < n) & (3 * KZ < n)


@pytest.mark.parametrize("n", [12, 24, 48, 96, 192])
def test_rhs_matches_oracle(fk, oracle_mod, n):
    u = _ic(oracle_mod, n, seed=n, k0=min(4.0, n / 8))
    plan = fk.fftk_plan_create(n, n, n)
    try:
        Ng = _rhs(fk, plan, u)
        Nf = _rhs(fk, plan, u, feps=0.1) if n == 48 else None
    finally:
        fk.fftk_plan_destroy(plan)
    uw = u.astype(np.complex128)
    assert rel_l2(Ng, oracle_mod.ns_rhs(uw)) < 1e-5
    assert not np.any(Ng[:, ~_kept(n)])
    if Nf is not None:
        assert rel_l2(Nf, oracle_mod.ns_rhs(uw, force_eps=0.1, force_k2=(1, 4))) < 1e-5


@pytest.mark.parametrize("scheme", ["rk2", "rk4"])
def test_steps_match_oracle(fk, oracle_mod, scheme):
    n, nu, dt, steps = 48, 1e-3, 1e-3, 5
    u0 = _ic(oracle_mod, n, seed=2, k0=3.0)
    plan = fk.fftk_plan_create(n, n, n)
    try:
        ud = to_dev_c64(u0)
        prm = fk.make_params(nu, dt, scheme=fk.TARANG_RK4 if scheme == "rk4" else fk.TARANG_RK2)
        E, eps, _ = fk.tarang_ns_step(plan, ud.data_ptr(), prm, steps, True, stream())
        ug = from_dev_c64(ud)
    finally:
        fk.fftk_plan_destroy(plan)
    step = oracle_mod.ns_step_rk4 if scheme == "rk4" else oracle_mod.ns_step
    uo = step(u0.astype(np.complex128), nu, dt, steps)
    Eo, epso, _ = oracle_mod.diag(uo, nu)
    assert rel_l2(ug, uo) < 1e-5
    assert abs(E - Eo) < 1e-6 * Eo and abs(eps - epso) < 1e-5 * epso


def test_taylor_green_exact_decay(fk, oracle_mod):
    n, nu, dt, steps = 96, 0.01, 1e-3, 20
    u0 = oracle_mod.ic_taylor_green(n).astype(np.complex64)
    plan = fk.fftk_plan_create(n, n, n)
    try:
        ud = to_dev_c64(u0)
        E, eps, _ = fk.tarang_ns_step(plan, ud.data_ptr(), fk.make_params(nu, dt), steps, True, stream())
    finally:
        fk.fftk_plan_destroy(plan)
    want = 0.25 * np.exp(-4 * nu * steps * dt)
    assert abs(E - want) < 2.4e-6 * 0.25
    assert abs(eps - 4 * nu * want) < 1e-5 * eps


def test_library_initial_field_matches_oracle(fk, oracle_mod):
    import torch

    n = 48
    normals = synth.normal_fields(4, 3, (n, n, n))
    plan = fk.fftk_plan_create(n, n, n)
    try:
        nr = torch.from_numpy(normals.astype(np.float32)).to("cuda:0")
        u = empty_c64((3, n, n, n // 2 + 1))
        fk.tarang_ic_random(plan, nr.data_ptr(), u.data_ptr(), 3.0, 0.5, stream())
        sync()
        ug = from_dev_c64(u)
    finally:
        fk.fftk_plan_destroy(plan)
    uo = oracle_mod.ic_random(normals.astype(np.float32).astype(np.float64), k0=3.0, E0=0.5)
    assert rel_l2(ug, uo) < 1e-5
    assert abs(oracle_mod.diag(ug.astype(np.complex128))[0] - 0.5) < 1e-6


def test_split16_plan_on_a_3x2m_grid(fk, oracle_mod):
    # the split-FP16 stages need power-of-two lines: a 3 * 2^m plan runs its
    # passes in FP32 and the unfused right-hand side
    n = 48
    u = _ic(oracle_mod, n, seed=6, k0=3.0)
    plan = fk.fftk_plan_create(n, n, n, fk.FFTK_R32_SPLIT16)
    try:
        Ng = _rhs(fk, plan, u)
    finally:
        fk.fftk_plan_destroy(plan)
    assert rel_l2(Ng, oracle_mod.ns_rhs(u.astype(np.complex128))) < 1e-5


def _embed(u, N):
    n = u.shape[1]
    a = np.arange(n)
    a = a[2 * a != n]
    big = np.where(2 * a < n, a, a - n + N)
    out = np.zeros((3, N, N, N // 2 + 1), dtype=u.dtype)
    for c in range(3):
        out[c][np.ix_(big, big, np.arange(n // 2 + 1))] = u[c][np.ix_(a, a, np.arange(n // 2 + 1))]
    return out


def test_rhs_768_band_limited_matches_oracle_at_512(fk, oracle_mod):
    u256 = _ic(oracle_mod, 256, seed=8, k0=32.0)
    No = oracle_mod.ns_rhs(_embed(u256, 512).astype(np.complex128))
    u768 = _embed(u256, 768)
    plan = fk.fftk_plan_create(768, 768, 768)
    try:
        Ng = _rhs(fk, plan, u768)
    finally:
        fk.fftk_plan_destroy(plan)
    del u768
    a = np.arange(512)
    rows = np.where(2 * a < 512, a, a - 512 + 768)  # the 512^3 grid's rows inside the 768^3 one
    sub = np.stack([Ng[c][np.ix_(rows, rows, np.arange(257))] for c in range(3)])
    rel = rel_l2(sub, No)
    inside = np.zeros(768, dtype=bool)
    inside[rows] = True
    out = 0.0
    for c in range(3):
        for i in range(768):
            row = Ng[c, i].astype(np.complex128)
            if inside[i]:
                out += float(np.sum(np.abs(row[~inside, :]) ** 2) + np.sum(np.abs(row[inside, 257:]) ** 2))
            else:
                out += float(np.sum(np.abs(row) ** 2))
    rel_out = np.sqrt(out) / np.linalg.norm(No.ravel())
    print(f"\nMEASURED rhs768 band-limited rel_l2 {rel:.3e} outside {rel_out:.3e}")
    assert rel < 1e-5 and rel_out < 1e-5
