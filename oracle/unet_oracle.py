"""FP64 CPU oracle of the conv U-Net forecast surrogate (forward and backward).

TEST INFRASTRUCTURE ONLY: the GPU BF16 training and inference kernels are
checked against it; nothing in the library imports it.

The surrogate replaces the paper's ViT (Sec. III-B) by a small convolutional
U-Net that maps one SQG state x_t [2][n][n] to the next, x_{t+Delta} =
x_t + net(x_t) (residual form).  Layout NHWC inside; the SQG domain is
doubly periodic, so every 3x3 convolution pads circularly.

Architecture for widths (c1, c2, c3, c4):
    enc1: conv(2->c1), conv(c1->c1)           at n
    pool; enc2: conv(c1->c2), conv(c2->c2)    at n/2
    pool; enc3: conv(c2->c3), conv(c3->c3)    at n/4
    pool; mid:  conv(c3->c4), conv(c4->c4)    at n/8
    up, concat enc3 -> conv(c4+c3->c3), conv(c3->c3)
    up, concat enc2 -> conv(c3+c2->c2), conv(c2->c2)
    up, concat enc1 -> conv(c2+c1->c1), conv(c1->c1)
    head: 1x1 conv (c1 -> 2), no activation; output = input + head
conv = 3x3 convolution + bias + SiLU (z sigmoid(z)); pool = 2x2 mean;
up = nearest-neighbour x2; concat order = [upsampled, skip].
Loss = mean of squared error.  Parameters in one flat vector, per layer
W [Cout][3][3][Cin] then b [Cout]; head W [2][c1] then b [2].
"""
from __future__ import annotations

import numpy as np


def layer_shapes(widths, in_ch=2, out_ch=2):
    c1, c2, c3, c4 = widths
    convs = [(in_ch, c1), (c1, c1), (c1, c2), (c2, c2), (c2, c3), (c3, c3), (c3, c4), (c4, c4),
             (c4 + c3, c3), (c3, c3), (c3 + c2, c2), (c2, c2), (c2 + c1, c1), (c1, c1)]
    return convs, (c1, out_ch)


def param_count(widths, in_ch=2, out_ch=2):
    convs, (hc, ho) = layer_shapes(widths, in_ch, out_ch)
    return sum(9 * ci * co + co for ci, co in convs) + hc * ho + ho


def init_params(widths, seed, in_ch=2, out_ch=2):
    """He-uniform weights, zero biases; the head starts small."""
    g = np.random.default_rng(seed)
    convs, (hc, ho) = layer_shapes(widths, in_ch, out_ch)
    parts = []
    for ci, co in convs:
        bound = np.sqrt(6.0 / (9 * ci))
        parts.append(g.uniform(-bound, bound, 9 * ci * co))
        parts.append(np.zeros(co))
    parts.append(g.uniform(-0.01, 0.01, hc * ho))
    parts.append(np.zeros(ho))
    return np.concatenate(parts).astype(np.float32)


def unpack(params, widths, in_ch=2, out_ch=2):
    convs, (hc, ho) = layer_shapes(widths, in_ch, out_ch)
    off = 0
    layers = []
    for ci, co in convs:
        W = params[off:off + 9 * ci * co].reshape(co, 3, 3, ci)
        off += 9 * ci * co
        b = params[off:off + co]
        off += co
        layers.append((W.astype(np.float64), b.astype(np.float64)))
    Wh = params[off:off + hc * ho].reshape(ho, hc).astype(np.float64)
    off += hc * ho
    bh = params[off:off + ho].astype(np.float64)
    return layers, (Wh, bh)


def _im2col(x):
    """x [B][H][W][C] -> [B][H][W][3*3*C], (dy, dx, c) order, circular padding."""
    cols = []
    for dy in range(3):
        for dx in range(3):
            cols.append(np.roll(np.roll(x, 1 - dy, axis=1), 1 - dx, axis=2))
    return np.concatenate(cols, axis=3)


def _col2im(dcol, C):
    """Adjoint of _im2col."""
    B, H, W, _ = dcol.shape
    dx_ = np.zeros((B, H, W, C))
    i = 0
    for dy in range(3):
        for dx in range(3):
            dx_ += np.roll(np.roll(dcol[..., i * C:(i + 1) * C], dy - 1, axis=1), dx - 1, axis=2)
            i += 1
    return dx_


def _sig(z):
    return 1.0 / (1.0 + np.exp(-z))


def _conv_fwd(x, W, b):
    col = _im2col(x)
    z = col @ W.reshape(W.shape[0], -1).T + b
    return z * _sig(z), (x, z)


def _conv_bwd(dy, cache, W):
    x, z = cache
    s = _sig(z)
    dz = dy * s * (1.0 + z * (1.0 - s))
    col = _im2col(x)
    dW = (dz.reshape(-1, dz.shape[-1]).T @ col.reshape(-1, col.shape[-1])).reshape(W.shape)
    db = dz.sum(axis=(0, 1, 2))
    dcol = dz @ W.reshape(W.shape[0], -1)
    return _col2im(dcol, x.shape[-1]), dW, db


def _pool(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def _pool_bwd(dy):
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) / 4.0


def _up(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def _up_bwd(dy):
    B, H, W, C = dy.shape
    return dy.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def forward(params, widths, x_nchw, with_cache=False):
    """x [B][2][n][n] -> prediction [B][2][n][n] (FP64)."""
    layers, (Wh, bh) = unpack(params, widths)
    x = np.transpose(np.asarray(x_nchw, dtype=np.float64), (0, 2, 3, 1))
    caches = []

    def conv(h, i):
        out, c = _conv_fwd(h, *layers[i])
        caches.append(c)
        return out

    e1 = conv(conv(x, 0), 1)
    e2 = conv(conv(_pool(e1), 2), 3)
    e3 = conv(conv(_pool(e2), 4), 5)
    m = conv(conv(_pool(e3), 6), 7)
    d3 = conv(conv(np.concatenate([_up(m), e3], axis=3), 8), 9)
    d2 = conv(conv(np.concatenate([_up(d3), e2], axis=3), 10), 11)
    d1 = conv(conv(np.concatenate([_up(d2), e1], axis=3), 12), 13)
    head = d1 @ Wh.T + bh
    out = x + head
    y = np.transpose(out, (0, 3, 1, 2))
    if with_cache:
        return y, dict(x=x, e1=e1, e2=e2, e3=e3, m=m, d3=d3, d2=d2, d1=d1, caches=caches)
    return y


def adamw_step(w, g, m, v, step, lr, weight_decay, beta1=0.9, beta2=0.999, eps=1e-8):
    """One AdamW update in FP64 (Loshchilov and Hutter, "Decoupled Weight
    Decay Regularization", ICLR 2019, their Algorithm 2 with the step size
    alpha = 1 and the schedule multiplier eta_t = lr):

        m_t = beta1 m_{t-1} + (1 - beta1) g_t
        v_t = beta2 v_{t-1} + (1 - beta2) g_t^2
        m^_t = m_t / (1 - beta1^t),   v^_t = v_t / (1 - beta2^t)
        w_t = w_{t-1} - lr (m^_t / (sqrt(v^_t) + eps) + weight_decay w_{t-1})

    The weight decay acts on the parameters directly (decoupled from the
    gradient-based step), not through the gradient as an L2 penalty would.
    ``step`` is t >= 1, the index of this update.  Returns (w_t, m_t, v_t)."""
    w = np.asarray(w, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** step)
    v_hat = v / (1.0 - beta2 ** step)
    w_new = w - lr * (m_hat / (np.sqrt(v_hat) + eps) + weight_decay * w)
    return w_new, m, v


def loss_and_grad(params, widths, x_nchw, target_nchw):
    """Mean-squared-error loss and its gradient with respect to the flat
    parameter vector (FP64, hand-written backward pass)."""
    layers, (Wh, bh) = unpack(params, widths)
    y, c = forward(params, widths, x_nchw, with_cache=True)
    t = np.asarray(target_nchw, dtype=np.float64)
    diff = y - t
    loss = float(np.mean(diff ** 2))
    dout = np.transpose(2.0 * diff / diff.size, (0, 2, 3, 1))
    grads_W = [None] * len(layers)
    grads_b = [None] * len(layers)
    caches = c["caches"]
    dWh = (dout.reshape(-1, dout.shape[-1]).T @ c["d1"].reshape(-1, c["d1"].shape[-1]))
    dbh = dout.sum(axis=(0, 1, 2))
    dd1 = dout @ Wh

    def back(dy, i):
        dx, dW, db = _conv_bwd(dy, caches[i], layers[i][0])
        grads_W[i], grads_b[i] = dW, db
        return dx

    c1 = c["e1"].shape[-1]
    c2 = c["e2"].shape[-1]
    c3 = c["e3"].shape[-1]
    g = back(back(dd1, 13), 12)
    d_up2, de1 = g[..., :g.shape[-1] - c1], g[..., g.shape[-1] - c1:]
    g = back(back(_up_bwd(d_up2), 11), 10)
    d_up3, de2 = g[..., :g.shape[-1] - c2], g[..., g.shape[-1] - c2:]
    g = back(back(_up_bwd(d_up3), 9), 8)
    d_upm, de3 = g[..., :g.shape[-1] - c3], g[..., g.shape[-1] - c3:]
    g = back(back(_up_bwd(d_upm), 7), 6)
    de3 = de3 + _pool_bwd(g)
    g = back(back(de3, 5), 4)
    de2 = de2 + _pool_bwd(g)
    g = back(back(de2, 3), 2)
    de1 = de1 + _pool_bwd(g)
    back(back(de1, 1), 0)
    parts = []
    for dW, db in zip(grads_W, grads_b):
        parts.append(dW.reshape(-1))
        parts.append(db)
    parts.append(dWh.reshape(-1))
    parts.append(dbh)
    return loss, np.concatenate(parts)
