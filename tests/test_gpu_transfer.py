"""GPU parity of the energy transfer spectrum T(K) and flux Pi(K)
(tarang_transfer) against the FP64 oracle, through the C ABI.

T(K) = sum over shell K of w Re(conj(u) . N) with N the FP32 right-hand
side.  The right-hand side is held to relative L2 1e-5 of the oracle's
(FP32 transforms; the error is spread over all modes, not proportional to
each shell's own content), so by Cauchy-Schwarz each shell's error is
bounded by 1e-5 ||u_K|| ||N|| (weighted norms, u over the shell, N over the
whole spectrum); the FP64 reduction adds nothing visible at that level.
"""
import numpy as np
import pytest

import synth
from gpu_helpers import to_dev_c64

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


def _stream():
    import torch

    return torch.cuda.current_stream(torch.device("cuda:0")).cuda_stream


def _shells_and_weights(n):
    a = np.arange(n)
    k = np.where(2 * a < n, a, a - n)
    KX, KY, KZ = np.meshgrid(k, k, np.arange(n // 2 + 1), indexing="ij")
    shell = np.floor(np.sqrt(KX**2 + KY**2 + KZ**2) + 0.5).astype(int)
    w = np.where((KZ == 0) | (2 * KZ == n), 1.0, 2.0)
    return shell, w


def _shell_norm_bound(u, N, n, nb):
    shell, w = _shells_and_weights(n)
    uu = np.sum(np.abs(u) ** 2, axis=0) * w
    eu = np.bincount(shell.ravel(), uu.ravel(), minlength=nb)[:nb]
    eN = np.sum(np.sum(np.abs(N) ** 2, axis=0) * w)
    return np.sqrt(eu * eN)


def _random_ic(oracle_mod, n, seed, k0):
    u = oracle_mod.ic_random(synth.normal_fields(seed, 3, (n, n, n)), k0=k0, E0=0.5)
    return u.astype(np.complex64)


@pytest.mark.parametrize("n", [16, 32, 64])
def test_transfer_spectrum_matches_oracle(fk, oracle_mod, n):
    u = _random_ic(oracle_mod, n, seed=100 + n, k0=min(4.0, n / 8))
    plan = fk.fftk_plan_create(n, n, n)
    try:
        ud = to_dev_c64(u)
        total, T, Pi = fk.tarang_transfer(plan, ud.data_ptr(), None, _stream())
        again = fk.tarang_transfer(plan, ud.data_ptr(), None, _stream())
    finally:
        fk.fftk_plan_destroy(plan)
    T, Pi = np.array(T), np.array(Pi)
    u64 = u.astype(np.complex128)
    N = oracle_mod.ns_rhs(u64)
    To = oracle_mod.transfer_spectrum(u64, N)
    assert len(T) == len(To)
    bound = 1e-5 * _shell_norm_bound(u64, N, n, len(T))
    assert np.all(np.abs(T - To) <= bound + 1e-300), np.max(np.abs(T - To) / (bound + 1e-300))
    assert np.max(np.abs(To)) > 1e2 * np.max(bound)  # the bound is far below the signal
    # flux is the running sum of -T in shell order; the total agrees with sum_K T
    assert np.array_equal(Pi, -np.cumsum(T))
    assert abs(total - T.sum()) <= 1e-12 * np.sum(np.abs(T))
    # conservation: the nonlinear term moves energy between shells only
    scale = np.sqrt(np.sum(np.abs(u64) ** 2) * np.sum(np.abs(N) ** 2)) * 2
    assert abs(total) < 1e-5 * scale
    # bitwise reproducible
    assert again[0] == total and list(again[1]) == list(T)


def test_transfer_of_forcing_lands_in_forced_shell(fk, oracle_mod):
    # forcing on 1 <= |k|^2 <= 2 (exactly shell 1) at power eps
    n, eps = 32, 0.1
    u = _random_ic(oracle_mod, n, seed=7, k0=2.0)
    plan = fk.fftk_plan_create(n, n, n)
    try:
        ud = to_dev_c64(u)
        _, T0, _ = fk.tarang_transfer(plan, ud.data_ptr(), None, _stream())
        tot, Tf, Pif = fk.tarang_transfer(plan, ud.data_ptr(), fk.make_params(0.0, 0.0, eps, (1, 2)), _stream())
    finally:
        fk.fftk_plan_destroy(plan)
    d = np.array(Tf) - np.array(T0)
    assert abs(d[1] - eps) < 1e-5 * eps
    assert np.max(np.abs(np.delete(d, 1))) < 1e-6 * np.max(np.abs(T0))
    assert abs(tot - eps) < 1e-5
    # all injected power leaves the sphere K = 1 or is held by the nonlinear flux
    assert abs(Pif[-1] + tot) < 1e-12 * np.sum(np.abs(Tf))


def test_transfer_full_size_matches_step_energy_budget(fk):
    # 512^3 field of the decaying workload after 100 steps.  One inviscid
    # step of dt changes each shell's energy by the trapezoid of T over the
    # step up to O(dt^3) (Heun): E_K(t+dt) - E_K(t) = dt/2 (T_K(t) + T_K(t+dt)).
    # This ties the transfer's shells and weights to the step and the
    # energy spectrum of tarang_diag at full size.  Also: conservation,
    # zero beyond the dealiased radius, bitwise repeat.
    import torch

    n, dt = 512, 1e-4
    dev = torch.device("cuda:0")
    st = _stream()
    plan = fk.fftk_plan_create(n, n, n)
    try:
        nr = torch.empty((3, n, n, n), dtype=torch.float32, device=dev)
        for f in range(3):
            fk.fftk_fill_normal(nr[f].data_ptr(), n**3, 20260, f, st)
        u = torch.empty((3, n, n, n // 2 + 1, 2), dtype=torch.float32, device=dev)
        fk.tarang_ic_random(plan, nr.data_ptr(), u.data_ptr(), 4.0, 0.5, st)
        del nr
        fk.tarang_ns_step(plan, u.data_ptr(), fk.make_params(1e-3, 5e-4), 100, False, st)
        tot, T0, Pi = fk.tarang_transfer(plan, u.data_ptr(), None, st)
        tot2, T0b, _ = fk.tarang_transfer(plan, u.data_ptr(), None, st)
        _, _, E0 = fk.tarang_diag(plan, u.data_ptr(), 0.0, st)
        fk.tarang_ns_step(plan, u.data_ptr(), fk.make_params(0.0, dt), 1, False, st)
        _, T1, _ = fk.tarang_transfer(plan, u.data_ptr(), None, st)
        _, _, E1 = fk.tarang_diag(plan, u.data_ptr(), 0.0, st)
    finally:
        fk.fftk_plan_destroy(plan)
    T0, T1, Pi = np.array(T0), np.array(T1), np.array(Pi)
    dE = np.array(E1) - np.array(E0)
    trap = 0.5 * dt * (T0 + T1)
    assert np.max(np.abs(trap)) > 0
    assert np.max(np.abs(dE - trap)) < 1e-3 * np.max(np.abs(trap)), np.max(np.abs(dE - trap))
    assert np.all(np.isfinite(T0))
    assert abs(tot) < 1e-5 * np.sum(np.abs(T0))
    assert T0[0] == 0.0 and Pi[0] == 0.0
    assert abs(Pi[-1]) < 1e-5 * np.sum(np.abs(T0))
    kd = (n - 1) // 3
    assert np.all(T0[int(np.ceil(np.sqrt(3) * kd)) + 1:] == 0)
    assert tot2 == tot and list(T0b) == list(T0)


def test_transfer_argument_errors(fk):
    plan = fk.fftk_plan_create(16, 16, 16)
    try:
        with pytest.raises(fk.FFTKError):
            fk.tarang_transfer(plan, 0, None, _stream())
    finally:
        fk.fftk_plan_destroy(plan)
    plan = fk.fftk_plan_create(16, 16, 32)
    try:
        import torch

        u = torch.zeros((3, 16, 16, 17, 2), dtype=torch.float32, device="cuda:0")
        with pytest.raises(fk.FFTKError):
            fk.tarang_transfer(plan, u.data_ptr(), None, _stream())
    finally:
        fk.fftk_plan_destroy(plan)


@pytest.mark.parametrize("n", [16, 32, 64])
def test_shell_transfer_matches_oracle(fk, oracle_mod, n):
    # T(r <- g) of FP32 transforms against the FP64 oracle: every entry within
    # 1e-5 of the largest (the FP32 transforms are good to ~1e-6 relative);
    # antisymmetry and the receivers' sums against tarang_transfer on the GPU
    u = _random_ic(oracle_mod, n, seed=200 + n, k0=min(4.0, n / 8))
    kmax = oracle_mod.kmax_shell(n)
    bounds = sorted({0, 1, 2, 3, 4, 6, n // 8, n // 4, n // 3, n // 2, kmax + 1})
    plan = fk.fftk_plan_create(n, n, n)
    try:
        ud = to_dev_c64(u)
        T = np.array(fk.tarang_shell_transfer(plan, ud.data_ptr(), bounds, _stream()))
        T2 = np.array(fk.tarang_shell_transfer(plan, ud.data_ptr(), bounds, _stream()))
        _, TK, _ = fk.tarang_transfer(plan, ud.data_ptr(), None, _stream())
    finally:
        fk.fftk_plan_destroy(plan)
    To = oracle_mod.shell_transfer(u.astype(np.complex128), bounds)
    scale = np.max(np.abs(To))
    assert scale > 1e-4
    assert np.max(np.abs(T - To)) < 1e-5 * scale, np.max(np.abs(T - To)) / scale
    assert np.array_equal(T, T2)
    assert np.max(np.abs(T + T.T)) < 2e-5 * scale
    TK = np.array(TK)
    rows = np.array([TK[bounds[i]:bounds[i + 1]].sum() for i in range(len(bounds) - 1)])
    assert np.max(np.abs(T.sum(axis=1) - rows)) < 2e-5 * scale


def test_shell_transfer_full_size_properties(fk):
    # 512^3 decaying-workload field after 100 steps, octave shells: the matrix
    # is antisymmetric, each receiver's givers add up to its T(K) from
    # tarang_transfer, and the flux through each bound equals the transfer
    # from the shells inside to those outside
    import torch

    n = 512
    dev = torch.device("cuda:0")
    st = _stream()
    plan = fk.fftk_plan_create(n, n, n)
    try:
        nr = torch.empty((3, n, n, n), dtype=torch.float32, device=dev)
        for f in range(3):
            fk.fftk_fill_normal(nr[f].data_ptr(), n**3, 20261, f, st)
        u = torch.empty((3, n, n, n // 2 + 1, 2), dtype=torch.float32, device=dev)
        fk.tarang_ic_random(plan, nr.data_ptr(), u.data_ptr(), 4.0, 0.5, st)
        del nr
        fk.tarang_ns_step(plan, u.data_ptr(), fk.make_params(1e-3, 5e-4), 100, False, st)
        kmax = fk.tarang_diag_kmax(plan)
        bounds = [0, 1, 2, 4, 8, 16, 32, 64, 128, 256, kmax + 1]
        T = np.array(fk.tarang_shell_transfer(plan, u.data_ptr(), bounds, st))
        _, TK, Pi = fk.tarang_transfer(plan, u.data_ptr(), None, st)
    finally:
        fk.fftk_plan_destroy(plan)
    TK, Pi = np.array(TK), np.array(Pi)
    scale = np.max(np.abs(T))
    assert np.all(np.isfinite(T)) and scale > 0
    assert np.max(np.abs(T + T.T)) < 1e-4 * scale
    rows = np.array([TK[bounds[i]:bounds[i + 1]].sum() for i in range(len(bounds) - 1)])
    assert np.max(np.abs(T.sum(axis=1) - rows)) < 1e-4 * scale
    for i in range(1, len(bounds) - 1):
        assert abs(T[i:, :i].sum() - Pi[bounds[i] - 1]) < 1e-4 * scale


def test_shell_transfer_argument_errors(fk):
    import torch

    plan = fk.fftk_plan_create(16, 16, 16)
    try:
        u = torch.zeros((3, 16, 16, 9, 2), dtype=torch.float32, device="cuda:0")
        kmax = fk.tarang_diag_kmax(plan)
        for bad in ([0, 2, 2], [3, 1], [-1, 2], [0, kmax + 2], [0]):
            with pytest.raises(fk.FFTKError):
                fk.tarang_shell_transfer(plan, u.data_ptr(), bad, _stream())
        # a zero field has zero transfer
        T = fk.tarang_shell_transfer(plan, u.data_ptr(), [0, 4, kmax + 1], _stream())
        assert np.array_equal(np.array(T), np.zeros((2, 2)))
    finally:
        fk.fftk_plan_destroy(plan)


def test_transfer_edge_cases(fk, oracle_mod):
    # one shell holding every mode: the matrix is the 1x1 transfer of the
    # whole field to itself, zero up to rounding; a split-FP16 plan gives the
    # spectrum of its own (unfused) right-hand side
    n = 32
    u = _random_ic(oracle_mod, n, seed=90, k0=3.0)
    plan = fk.fftk_plan_create(n, n, n)
    plan16 = fk.fftk_plan_create(n, n, n, fk.FFTK_R32_SPLIT16)
    try:
        ud = to_dev_c64(u)
        kmax = fk.tarang_diag_kmax(plan)
        T1 = np.array(fk.tarang_shell_transfer(plan, ud.data_ptr(), [0, kmax + 1], _stream()))
        Tfine = np.array(fk.tarang_shell_transfer(plan, ud.data_ptr(), [0, 2, 4, 8, kmax + 1], _stream()))
        _, TK, _ = fk.tarang_transfer(plan, ud.data_ptr(), None, _stream())
        _, TK16, _ = fk.tarang_transfer(plan16, ud.data_ptr(), None, _stream())
    finally:
        fk.fftk_plan_destroy(plan)
        fk.fftk_plan_destroy(plan16)
    assert T1.shape == (1, 1)
    assert abs(T1[0, 0]) < 1e-5 * np.max(np.abs(Tfine))
    TK, TK16 = np.array(TK), np.array(TK16)
    bound = 3e-5 * _shell_norm_bound(u.astype(np.complex128), oracle_mod.ns_rhs(u.astype(np.complex128)), n,
                                     len(TK))
    assert np.all(np.abs(TK16 - TK) <= bound + 1e-300)
