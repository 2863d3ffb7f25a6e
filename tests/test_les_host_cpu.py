"""Host-side logic of the closure workflow (paper_1805_07801_gb300/les.py):
the training-set normalisation, the flux weighting of the loss, the per-shell
comparison against the reference spectrum, and the configuration's data sets.
No GPU: these are plain numpy functions."""
import dataclasses

import numpy as np
import pytest

les = pytest.importorskip("paper_1805_07801_gb300.les")


def test_normalisation_whitens_inputs_and_scales_outputs_by_their_rms():
    rng = np.random.default_rng(0)
    inv = rng.normal(loc=[[3.0], [-2.0], [0.0], [10.0], [-5.0]], scale=[[1.0], [0.5], [2.0], [4.0], [0.1]],
                     size=(5, 20000))
    taup = rng.normal(scale=[[0.1], [0.2], [0.3], [0.05], [0.01], [1.0]], size=(6, 20000))
    shift, scale, out_scale = les.normalisation(inv, taup)
    x = (inv.T - shift) * scale
    assert np.allclose(x.mean(axis=0), 0.0, atol=1e-12)
    assert np.allclose(x.std(axis=0), 1.0, rtol=1e-12)
    assert np.allclose(np.sqrt(np.mean((taup.T / out_scale) ** 2, axis=0)), 1.0, rtol=1e-12)


def test_flux_weight_multiplies_the_diagonal_errors():
    # a weight w divides the diagonal components' scale by sqrt(w), so their
    # squared normalised errors grow by w and the off-diagonal ones do not change
    rng = np.random.default_rng(1)
    inv = rng.normal(size=(5, 1000))
    taup = rng.normal(size=(6, 1000))
    _, _, s1 = les.normalisation(inv, taup, 1.0)
    _, _, s4 = les.normalisation(inv, taup, 4.0)
    err = rng.normal(size=6)
    r = (err / s4) ** 2 / (err / s1) ** 2
    assert np.allclose(r[:3], 4.0) and np.allclose(r[3:], 1.0)


def test_constant_inputs_keep_finite_scales():
    shift, scale, out_scale = les.normalisation(np.ones((5, 10)), np.zeros((6, 10)))
    assert np.all(np.isfinite(scale)) and np.all(np.isfinite(out_scale)) and np.all(out_scale > 0)


def test_shell_comparison():
    ref = np.array([9.0, 1.0, 2.0, 4.0, 8.0])
    EK = np.array([0.0, 1.04, 1.8, 4.0, 9.0])
    out = les._compare(EK, ref, 4)
    assert np.allclose(out["shell_rel_err"], [0.04, 0.1, 0.0, 0.125])
    assert out["shells_within_5pct"] == 2
    assert out["max_rel_err"] == pytest.approx(0.125)
    assert out["mean_rel_err"] == pytest.approx((0.04 + 0.1 + 0.0 + 0.125) / 4)
    assert out["EK"] == EK.tolist()


def test_configurations():
    full = les.ClosureConfig()
    small = les.ClosureConfig.small()
    assert full.factor == 8 and small.factor == 8
    assert full.targets[0] == "box" and "les" in full.targets and "blend" in full.targets
    assert full.seeded_runs == 0 and small.targets == ("box",)
    assert dataclasses.replace(full, seeded_runs=8).seeded_targets == ("box", "blend")
