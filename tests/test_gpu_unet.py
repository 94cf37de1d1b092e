"""The BF16 U-Net surrogate kernels against the FP64 U-Net oracle: forward
output, loss, and the gradient of every parameter tensor (relative L2
<= 2e-2, the BF16 bar), then a short AdamW run that lowers the loss."""
import numpy as np
import pytest

from oracle import unet_oracle as uo

pytestmark = pytest.mark.gpu

WIDTHS = (8, 16, 16, 24)


def _segments(widths):
    convs, (hc, ho) = uo.layer_shapes(widths)
    segs, off = [], 0
    for ci, co in convs:
        segs.append(("W", off, off + 9 * ci * co))
        off += 9 * ci * co
        segs.append(("b", off, off + co))
        off += co
    segs.append(("Wh", off, off + hc * ho))
    off += hc * ho
    segs.append(("bh", off, off + ho))
    return segs


def test_unet_forward_and_gradients_match_oracle():
    import torch
    from paper_2407_12168_gb300 import ensf
    g = np.random.default_rng(0)
    params = uo.init_params(WIDTHS, seed=3)
    params[-(WIDTHS[0] * 2 + 2):] = g.uniform(-0.2, 0.2, WIDTHS[0] * 2 + 2).astype(np.float32)
    x = g.standard_normal((2, 2, 32, 32)).astype(np.float32)
    t = (x + 0.3 * g.standard_normal(x.shape)).astype(np.float32)
    net = ensf.UNet(WIDTHS, 32, 32, max_batch=2)
    assert net.nparams == params.size == uo.param_count(WIDTHS)
    net.set_params(torch.from_numpy(params).cuda())
    y = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    y_ref = uo.forward(params, WIDTHS, x)
    assert np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref) < 1e-2
    grad, loss = net.gradients(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    grad = grad.cpu().numpy()
    loss_ref, grad_ref = uo.loss_and_grad(params, WIDTHS, x, t)
    assert float(loss.item()) == pytest.approx(loss_ref, rel=1e-2)
    for name, a, b in _segments(WIDTHS):
        gr = grad_ref[a:b]
        err = np.linalg.norm(grad[a:b] - gr) / max(np.linalg.norm(gr), 1e-30)
        assert err <= 2e-2, (name, a, err)


def test_unet_training_lowers_the_loss():
    import torch
    from paper_2407_12168_gb300 import ensf
    g = np.random.default_rng(1)
    net = ensf.UNet(WIDTHS, 32, 32, max_batch=4)
    net.set_params(torch.from_numpy(uo.init_params(WIDTHS, seed=4)).cuda())
    x = torch.from_numpy(g.standard_normal((4, 2, 32, 32)).astype(np.float32)).cuda()
    # a smooth, learnable map: a shifted copy of the input
    t = torch.roll(x, shifts=1, dims=3) * 0.8
    first = float(net.train_step(x, t, lr=3e-3).item())
    for _ in range(60):
        last = float(net.train_step(x, t, lr=3e-3).item())
    assert last < 0.5 * first


def test_adamw_step_matches_oracle():
    """Two AdamW steps of ensf_unet_train_step against the oracle's FP64
    AdamW update applied to the same gradients: the FP32 master weights and
    both moments after each step.  The update (w_t - w_{t-1}) must agree to
    1e-5 relative; the stored weights then differ from the oracle's only by
    FP32 rounding of w_t itself."""
    import torch
    from paper_2407_12168_gb300 import ensf
    g = np.random.default_rng(5)
    params = uo.init_params(WIDTHS, seed=6)
    params[-(WIDTHS[0] * 2 + 2):] = g.uniform(-0.2, 0.2, WIDTHS[0] * 2 + 2).astype(np.float32)
    net = ensf.UNet(WIDTHS, 32, 32, max_batch=2)
    net.set_params(torch.from_numpy(params).cuda())
    lr, wd = 1e-2, 0.05
    w_prev = params.astype(np.float64)
    m_prev = np.zeros_like(w_prev)
    v_prev = np.zeros_like(w_prev)
    u32 = np.finfo(np.float32).eps
    for step in (1, 2):
        x = g.standard_normal((2, 2, 32, 32)).astype(np.float32)
        t = (x + 0.3 * g.standard_normal(x.shape)).astype(np.float32)
        xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
        # the gradient the step will use (the backward pass is deterministic)
        grad_a, _ = net.gradients(xd, td)
        grad_b, _ = net.gradients(xd, td)
        grad = grad_a.cpu().numpy().astype(np.float64)
        assert np.array_equal(grad, grad_b.cpu().numpy().astype(np.float64))
        net.train_step(xd, td, lr=lr, weight_decay=wd)
        w_gpu = net.get_params().cpu().numpy().astype(np.float64)
        m_gpu, v_gpu, nsteps = net.get_moments()
        m_gpu = m_gpu.cpu().numpy().astype(np.float64)
        v_gpu = v_gpu.cpu().numpy().astype(np.float64)
        assert nsteps == step
        w_ref, m_ref, v_ref = uo.adamw_step(w_prev, grad, m_prev, v_prev, step, lr, wd)
        # 1e-5 relative, plus the rounding of the kernel's own FP32 sums: where
        # beta1 m + (1 - beta1) g nearly cancels, a few units in the last place
        # of its two terms exceed 1e-5 of the small result
        m_round = 4 * u32 * (0.9 * np.abs(m_prev) + 0.1 * np.abs(grad))
        v_round = 4 * u32 * (0.999 * v_prev + 0.001 * grad * grad)
        for name, got, want, rnd in (("m", m_gpu, m_ref, m_round), ("v", v_gpu, v_ref, v_round)):
            err = np.abs(got - want)
            bnd = 1e-5 * np.abs(want) + rnd
            worst = int(np.argmax(err - bnd))
            assert np.all(err <= bnd), (step, name, worst, got[worst], want[worst])
        c1, c2 = 1.0 - 0.9 ** step, 1.0 - 0.999 ** step
        dw = w_ref - w_prev
        # the update to 1e-5, beyond what the moment rounding above and the
        # FP32 evaluation of the update and of w itself carry
        m_part = lr * (m_round / c1) / (np.sqrt(v_ref / c2) + 1e-8)
        bound = 1e-5 * np.abs(dw) + 8 * u32 * np.abs(dw) + 2 * u32 * np.abs(w_ref) + m_part
        upd_err = np.abs(w_gpu - w_ref)
        worst = int(np.argmax(upd_err - bound))
        assert np.all(upd_err <= bound), (step, worst, w_prev[worst], w_gpu[worst], w_ref[worst])
        # and the bound is tight: most updates agree far below it
        assert np.median(upd_err / np.maximum(np.abs(dw), 1e-30)) < 1e-5
        # continue from the GPU's own FP32 state, as the next kernel step does
        w_prev, m_prev, v_prev = w_gpu, m_gpu, v_gpu


@pytest.mark.parametrize("widths,grid", [((32, 32, 64, 64), 32), ((32, 64, 64, 96), 64),
                                         ((32, 64, 128, 192), 128)])
def test_implicit_convolutions_match_oracle(widths, grid):
    """Channel widths that are multiples of 32 run the 3x3 convolutions as
    implicit GEMMs (haloed input read tap by tap by TMA, bias and SiLU in the
    epilogue; the data gradients the same kernel with mirrored taps) wherever
    a 128-pixel tile holds whole image rows, and their weight gradients as
    nine GEMMs over the pixels of column-shifted input copies wherever image
    rows are at least 32 wide (32- and 64-pixel k-blocks; the 320-channel
    decoder input of the third case in two channel tiles); the smallest
    levels and the 2-channel input convolution keep the im2col form.  Output,
    loss and every parameter gradient against the FP64 oracle at the BF16
    bar."""
    import torch
    from paper_2407_12168_gb300 import ensf
    g = np.random.default_rng(9)
    params = uo.init_params(widths, seed=10)
    params[-(widths[0] * 2 + 2):] = g.uniform(-0.2, 0.2, widths[0] * 2 + 2).astype(np.float32)
    x = g.standard_normal((2, 2, grid, grid)).astype(np.float32)
    t = (x + 0.3 * g.standard_normal(x.shape)).astype(np.float32)
    net = ensf.UNet(widths, grid, grid, max_batch=2)
    net.set_params(torch.from_numpy(params).cuda())
    y = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    y_ref = uo.forward(params, widths, x)
    assert np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref) < 1e-2
    grad, loss = net.gradients(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    grad = grad.cpu().numpy()
    loss_ref, grad_ref = uo.loss_and_grad(params, widths, x, t)
    assert float(loss.item()) == pytest.approx(loss_ref, rel=1e-2)
    for name, a, b in _segments(widths):
        gr = grad_ref[a:b]
        err = np.linalg.norm(grad[a:b] - gr) / max(np.linalg.norm(gr), 1e-30)
        assert err <= 2e-2, (name, a, err)
