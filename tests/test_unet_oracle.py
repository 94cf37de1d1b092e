"""Pins of the FP64 U-Net oracle: hand-written gradients against central
finite differences of the loss, and the residual identity at zero head."""
import numpy as np
import pytest

from oracle import unet_oracle as uo

W = (3, 4, 4, 5)


def test_gradient_matches_finite_differences():
    g = np.random.default_rng(0)
    p = uo.init_params(W, seed=1).astype(np.float64)
    p[-(W[0] * 2 + 2):] = g.uniform(-0.3, 0.3, W[0] * 2 + 2)  # a non-trivial head
    x = g.standard_normal((2, 2, 16, 16))
    t = g.standard_normal((2, 2, 16, 16))
    loss, grad = uo.loss_and_grad(p, W, x, t)
    assert grad.shape == p.shape
    idx = g.choice(p.size, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (uo.loss_and_grad(p + e, W, x, t)[0] - uo.loss_and_grad(p - e, W, x, t)[0]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, grad[i])


def test_zero_head_is_identity():
    p = uo.init_params(W, seed=2)
    p[-(W[0] * 2 + 2):] = 0.0
    x = np.random.default_rng(3).standard_normal((1, 2, 16, 16))
    np.testing.assert_allclose(uo.forward(p, W, x), x, rtol=0, atol=0)


def test_param_count_of_the_surrogate():
    assert 1.8e6 < uo.param_count((32, 64, 128, 256)) < 2.2e6


def test_conv_forward_matches_direct_circular_convolution():
    """The oracle's im2col convolution against the definition written out as
    nested loops: z[b][h][w][o] = bias[o] + sum over dy, dx in {0, 1, 2} and
    input channels c of W[o][dy][dx][c] * x[b][(h + dy - 1) mod H][(w + dx - 1) mod W][c]
    (3x3 cross-correlation centred on tap (1, 1), periodic boundaries).
    Non-square, odd sizes so that a swapped axis or a wrong roll sign fails."""
    g = np.random.default_rng(7)
    B, H, Wd, ci, co = 2, 5, 7, 3, 4
    x = g.standard_normal((B, H, Wd, ci))
    Wt = g.standard_normal((co, 3, 3, ci))
    bias = g.standard_normal(co)
    out, (x_cache, z) = uo._conv_fwd(x, Wt, bias)
    ref = np.zeros((B, H, Wd, co))
    for b in range(B):
        for h in range(H):
            for w in range(Wd):
                for o in range(co):
                    acc = bias[o]
                    for dy in range(3):
                        for dx in range(3):
                            for c in range(ci):
                                acc += Wt[o, dy, dx, c] * x[b, (h + dy - 1) % H, (w + dx - 1) % Wd, c]
                    ref[b, h, w, o] = acc
    np.testing.assert_allclose(z, ref, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(out, ref / (1.0 + np.exp(-ref)), rtol=1e-13, atol=1e-13)
    assert x_cache is x


def test_adamw_first_and_second_step_by_hand():
    """Two AdamW updates of one parameter, worked out by hand from the
    published update (bias-corrected moments, decoupled weight decay):
    w0 = 1, lr = 0.1, weight decay 0.01, g1 = 0.5, g2 = -0.25.
    Step 1: m = 0.05, v = 0.00025, m^ = 0.5, v^ = 0.25,
            w1 = 1 - 0.1 (0.5 / (0.5 + 1e-8) + 0.01 * 1).
    Step 2: m = 0.9 * 0.05 - 0.1 * 0.25 = 0.02,
            v = 0.999 * 0.00025 + 0.001 * 0.0625 = 0.00031225,
            m^ = 0.02 / 0.19, v^ = 0.00031225 / 0.001999,
            w2 = w1 - 0.1 (m^ / (sqrt(v^) + 1e-8) + 0.01 w1)."""
    w1, m1, v1 = uo.adamw_step(np.array([1.0]), np.array([0.5]), np.zeros(1), np.zeros(1), 1, 0.1, 0.01)
    assert m1[0] == pytest.approx(0.05, rel=1e-15)
    assert v1[0] == pytest.approx(0.00025, rel=1e-14)
    w1_hand = 1.0 - 0.1 * (0.5 / (0.5 + 1e-8) + 0.01)
    assert w1[0] == pytest.approx(w1_hand, rel=1e-15)
    w2, m2, v2 = uo.adamw_step(w1, np.array([-0.25]), m1, v1, 2, 0.1, 0.01)
    assert m2[0] == pytest.approx(0.02, rel=1e-14)
    assert v2[0] == pytest.approx(0.00031225, rel=1e-14)
    mh, vh = 0.02 / 0.19, 0.00031225 / 0.001999
    w2_hand = w1_hand - 0.1 * (mh / (np.sqrt(vh) + 1e-8) + 0.01 * w1_hand)
    assert w2[0] == pytest.approx(w2_hand, rel=1e-14)
    # the first moment is still positive after the opposite gradient, so the
    # second update keeps the direction of the first (momentum)
    assert w2[0] < w1[0]


def test_adamw_constant_gradient_and_pure_decay():
    """Closed forms: with a constant gradient g the bias-corrected moments
    are exactly g and g^2 at every step, so each update moves the weight by
    lr * g / (|g| + eps) plus the decay; with g = 0 only the decoupled decay
    acts, w_T = w_0 (1 - lr * lambda)^T (an L2 penalty folded into the
    gradient would instead be normalised by sqrt(v^) and move w by about lr
    per step)."""
    g = np.array([0.3, -2.0, 1e-3])
    w = np.array([0.5, -0.1, 2.0])
    m = np.zeros(3)
    v = np.zeros(3)
    lr, lam = 1e-2, 0.0
    for t in range(1, 8):
        w_prev = w
        w, m, v = uo.adamw_step(w, g, m, v, t, lr, lam)
        np.testing.assert_allclose(w_prev - w, lr * g / (np.abs(g) + 1e-8), rtol=1e-12)
    w0 = np.array([1.5, -3.0])
    w, m, v = w0, np.zeros(2), np.zeros(2)
    for t in range(1, 11):
        w, m, v = uo.adamw_step(w, np.zeros(2), m, v, t, 0.05, 0.2)
    np.testing.assert_allclose(w, w0 * (1.0 - 0.05 * 0.2) ** 10, rtol=1e-14)
