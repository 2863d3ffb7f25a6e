"""The Navier-Stokes step of a FFTK_R32_SPLIT16 plan: the right-hand side is
evaluated unfused through the library's transforms, whose radix-16 stages run
on the tensor cores (split FP16 hi/lo operands, FP32 accumulation).

Tolerance: each of the nine transforms of a right-hand side carries the split
mode's ~2e-6 relative error (against ~3e-7 in FP32), so the right-hand side is
held to relative L2 3e-5 against the FP64 oracle; a few steps of the split and
the FP32 run of the same state stay within 1e-5 of each other.
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
    sync()
    return from_dev_c64(nd)


@pytest.mark.parametrize("n", [256])
def test_split16_rhs_matches_oracle(fk, oracle_mod, n):
    u = _ic(oracle_mod, n, seed=11, k0=4.0)
    plan = fk.fftk_plan_create(n, n, n, fk.FFTK_R32_SPLIT16)
    try:
        Ng = _rhs(fk, plan, u)
        Nf = _rhs(fk, plan, u, feps=0.1)
    finally:
        fk.fftk_plan_destroy(plan)
    No = oracle_mod.ns_rhs(u.astype(np.complex128))
    assert rel_l2(Ng, No) < 3e-5
    # constant-power forcing injects exactly eps (energy transfer of the forced term)
    assert abs(oracle_mod.transfer(u.astype(np.complex128), Nf) - 0.1) < 1e-4


def test_split16_steps_track_fp32(fk, oracle_mod):
    n = 256
    u = _ic(oracle_mod, n, seed=12, k0=4.0)
    out = {}
    for dt_name, dtype in (("fp32", fk.FFTK_R32), ("split16", fk.FFTK_R32_SPLIT16)):
        plan = fk.fftk_plan_create(n, n, n, dtype)
        try:
            ud = to_dev_c64(u)
            d = fk.tarang_ns_step(plan, ud.data_ptr(), fk.make_params(1e-3, 5e-4, 0.1, (1, 4)), 5, True, stream())
            out[dt_name] = (from_dev_c64(ud), d)
        finally:
            fk.fftk_plan_destroy(plan)
    (u32, d32), (u16, d16) = out["fp32"], out["split16"]
    assert rel_l2(u16, u32) < 1e-5
    assert abs(d16[0] - d32[0]) < 1e-6 * d32[0]
    assert abs(d16[1] - d32[1]) < 1e-5 * d32[1]
