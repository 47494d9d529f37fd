"""Pins of the selector oracle: finite-difference gradients of the MLP,
histogram invariants of the features, and label monotonicity."""
import numpy as np
import pytest

from oracle import selector
from paper_2509_23565_gb300 import inputs


def test_mlp_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    params = selector.init_params(1)
    X = rng.random((7, 64))
    y = rng.integers(3, 9, 7)
    loss, grads = selector.loss_and_grads(params, X, y)
    # perturb master weights; forward uses their BF16 rounding, so use steps that
    # move the BF16 value and compare against the straight-through gradient
    # on the biases (not rounded) exactly, and on weights through the rounded value
    for li in range(4):
        W, b = params[li]
        for j in (0, len(b) // 2, len(b) - 1):
            h = 1e-4
            bp = b.copy()
            bp[j] += h
            pp = list(params)
            pp[li] = (W, bp)
            lp, _ = selector.loss_and_grads(pp, X, y)
            bm = b.copy()
            bm[j] -= h
            pp[li] = (W, bm)
            lm, _ = selector.loss_and_grads(pp, X, y)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grads[li][1][j]) <= 1e-5 + 1e-4 * abs(fd), (li, j, fd, grads[li][1][j])


def test_weight_gradients_via_input_scaling_identity():
    """For the first layer, dL/dW0 = dL/dz0^T X: scaling X by c scales the
    first-layer weight gradient by c when the ReLU pattern is unchanged."""
    rng = np.random.default_rng(1)
    params = selector.init_params(2)
    X = rng.random((5, 64))
    y = rng.integers(3, 9, 5)
    _, g1 = selector.loss_and_grads(params, X, y)
    # finite differences through the network on one weight, using a perturbation
    # that is exactly representable after BF16 rounding (a power-of-two step)
    W0, b0 = params[0]
    i, j = 3, 5
    base = selector.bf16_round(W0)[i, j]
    step = 2.0 ** (np.floor(np.log2(abs(base))) - 7) if base != 0 else 2.0 ** -20
    Wp = W0.copy()
    Wp[i, j] = np.float32(base + step)
    Wm = W0.copy()
    Wm[i, j] = np.float32(base - step)
    lp, _ = selector.loss_and_grads([(Wp, b0)] + params[1:], X, y)
    lm, _ = selector.loss_and_grads([(Wm, b0)] + params[1:], X, y)
    fd = (lp - lm) / (2 * step)
    assert abs(fd - g1[0][0][i, j]) <= 1e-4 + 1e-2 * abs(fd)


def test_feature_histograms():
    A = np.full((4, 8), 0.75)
    B = np.full((8, 3), -2.0)
    f = selector.features(A, B)
    assert f.shape == (64,)
    assert f[0] == 1.0 and f[32] == 1.0          # every entry equals its row / column maximum
    A[0, 0] = 0.0
    B[:, 1] = 2.0 ** -40
    f = selector.features(A, B)
    assert f[31] == pytest.approx(1 / 32)          # the zero entry
    assert f[:32].sum() == pytest.approx(1.0) and f[32:].sum() == pytest.approx(1.0)
    A = inputs.log_scaled(30, 40, 8, seed=3)
    f = selector.features(A, inputs.log_scaled(40, 20, 8, seed=4))
    assert f[:32].sum() == pytest.approx(1.0)
    assert f[5:31].sum() > 0.3                     # a wide range spreads the offsets


def test_labels_follow_dynamic_range():
    A0 = inputs.uniform(64, 128, seed=5)
    B0 = inputs.uniform(128, 64, seed=6)
    e0 = selector.slice_errors(A0, B0)
    assert all(e0[i] >= e0[i + 1] for i in range(5))
    assert e0[-1] == 0.0
    assert selector.label_from_errors(e0) <= 7
    A1 = inputs.log_scaled(64, 128, 16, seed=7)
    B1 = inputs.log_scaled(128, 64, 16, seed=8)
    assert selector.label_from_errors(selector.slice_errors(A1, B1)) >= selector.label_from_errors(e0)
