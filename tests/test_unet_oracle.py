"""Pins of the FP64 U-Net oracle: hand-written gradients against central
finite differences of the loss, and the residual identity at zero head."""
import numpy as np

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
