"""What the trained initialiser gains over the method without it (the plain voxel-PCA /
heuristic cascade): on a scene not used for training, the MLP's predicted residuals
(optimised minus initial Gaussian parameters) must be closer to the residuals the plain
mapping loop actually produces than the zero residual of the plain initialisation is."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_trained_initialiser_predicts_heldout_residuals():
    from paper_2604_12942_gb300 import learned_init as li
    n = 40_000
    x, y = li.training_pairs([10, 11], n, iters=150, views=8)
    mlp, losses = li.train_mlp(x, y, epochs=30)
    assert losses[-1] < losses[0]
    xh, yh = li.training_pairs([20], n, iters=150, views=8)   # held-out scene
    pred = mlp.infer(xh)
    torch.cuda.synchronize()
    used = slice(0, 11)
    err_plain = float((yh[:, used] ** 2).mean())
    err_model = float(((pred[:, used] - yh[:, used]) ** 2).mean())
    print(f"held-out residual MSE: plain init {err_plain:.5f}, learned init {err_model:.5f}")
    assert np.isfinite(err_model)
    assert err_model < 0.9 * err_plain, (err_plain, err_model)
