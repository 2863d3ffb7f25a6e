"""What the trained closure gains over the coarse method without it.

The whole workflow at reduced size (256^3 forced resolved run, factor-8 box
filter to 32^3, 3000 training steps, 5000 coarse steps): the network must
beat a zero prediction on the held-out snapshot, and the coarse run with the
fused model must track the filtered resolved spectrum much better than the
same run without it (mean per-shell relative error over shells 1..10).
"""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def result():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_07801_gb300 import build as b

    b.build()
    from paper_1805_07801_gb300 import les

    return les.run(les.ClosureConfig.small(), log=None)


def test_network_beats_zero_model_on_heldout_snapshot(result):
    assert result["heldout_loss"] < 0.85 * result["heldout_loss_zero_model"]


def test_coarse_runs_stay_finite(result):
    assert result["model"]["finite"] and result["no_model"]["finite"]


@pytest.mark.parametrize("window", ["stated", "long"])
def test_model_gains_over_no_model(result, window):
    with_model = result["model"][window]["mean_rel_err"]
    without = result["no_model"][window]["mean_rel_err"]
    assert with_model < 0.5 * without, (with_model, without)


def test_coarse_run_is_faster_than_resolved(result):
    assert result["speedup"] > 1.0
