"""End-to-end learned indicator on solver-generated data (small sizes):
labels from the plain TVB detector on seeded blasts, training with the
library's kernels, then the gated run against the plain run on the 128^3
blast in the FP32 form. The gain shown is the limiter time: the TVB procedure
runs only on flagged cells."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_indicator_pipeline_and_gain():
    import torch
    from paper_1806_02343_gb300 import indicator as I
    X, y, nin, src = I.generate("powell", 2, n=32, seeds=(1, 2, 3), steps=5)
    assert X.shape[0] == 3 * 5 * 32 ** 3 and int(y.sum()) > 100 and int(src.sum()) == 0
    theta, info = I.train(X, y, nin, epochs=20, batch=1024, lr=2e-3, src=src)
    assert info["loss_last_epoch"] < 0.5 * info["loss_initial"]
    from paper_1806_02343_gb300.binding import DG_PREC_FP32MIX
    # the benchmarked form and size class: FP32 form at 128^3 (the staged
    # tensor-core indicator; x-rows of whole 128-cell tiles)
    rep = I.evaluate(theta, nin, "powell", 2, n=128, steps=4, threshold=0.1, precision=DG_PREC_FP32MIX)
    assert rep["status"]["plain"] == 0 and rep["status"]["mlp"] == 0
    assert rep["troubled_plain"] > 0
    assert rep["missed_cell_rate"] < 0.3
    assert rep["false_positive_rate"] < 0.1
    # the gain: network + TVB on flagged cells is cheaper than TVB detection on every cell
    assert rep["limiter_ms"]["mlp"] < rep["limiter_ms"]["plain"]
    # shocked runs: the density stays close; the other L1 differences are reported
    assert rep["l1_rel_final_means"][0] < 1e-3


def test_turbulence_samples():
    """Turbulence sources: every troubled cell kept and a share `keep` of the others."""
    from paper_1806_02343_gb300 import indicator as I
    X, y, nin, src = I.generate("glm", 2, seeds=(), turbulence=((32, 4.0, 11, 0.5),), turb_steps=2, turb_every=4)
    nt = X.shape[0]
    assert int(src.sum()) == nt and X.shape[1] >= nin
    assert 0.4 * 2 * 32 ** 3 < nt < 2 * 32 ** 3
    assert int(y.sum()) <= nt
