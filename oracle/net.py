"""The learned basis surrogate's network, written plainly in float64 numpy:
3x3x3 convolutions with zero padding (cross-correlation, output size =
input size), ReLU, the masked mean-squared error and one Adam step
(Kingma and Ba, 2015).  Used to check the GPU layer kernels' forward
values and gradients.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Layout: activations (B, C, S, S, S) with axes (batch, channel, z, y, x);
weights (co, ci, 27) with tap t = (dx+1) + 3 (dy+1) + 9 (dz+1).
"""
from __future__ import annotations

import numpy as np

TAPS = [(t % 3 - 1, (t // 3) % 3 - 1, t // 9 - 1) for t in range(27)]   # (dx, dy, dz)


def shifted(x, dx, dy, dz):
    """s[..., z, y, x] = x[..., z+dz, y+dy, x+dx], zero outside."""
    S = x.shape[-1]
    out = np.zeros_like(x)
    zs = slice(max(0, -dz), S - max(0, dz))
    ys = slice(max(0, -dy), S - max(0, dy))
    xs = slice(max(0, -dx), S - max(0, dx))
    zt = slice(max(0, dz), S - max(0, -dz))
    yt = slice(max(0, dy), S - max(0, -dy))
    xt = slice(max(0, dx), S - max(0, -dx))
    out[..., zs, ys, xs] = x[..., zt, yt, xt]
    return out


def conv_forward(x, w, b, relu):
    """y[b, o, v] = bias[o] + sum_i sum_t w[o, i, t] x[b, i, v + d(t)]."""
    B, ci = x.shape[:2]
    co = w.shape[0]
    y = np.zeros((B, co) + x.shape[2:])
    for t, (dx, dy, dz) in enumerate(TAPS):
        xs = shifted(x, dx, dy, dz)                       # (B, ci, S, S, S)
        y += np.einsum("oi,bizyx->bozyx", w[:, :, t], xs)
    y += b[None, :, None, None, None]
    return np.maximum(y, 0.0) if relu else y


def conv_backward(x, w, gy):
    """Gradients of L with respect to x, w and b given gy = dL/dy (y the
    pre-activation output): gx[b, i, u] = sum_o sum_t w[o, i, t] gy[b, o, u - d(t)],
    gw[o, i, t] = sum_b sum_v gy[b, o, v] x[b, i, v + d(t)], gb[o] = sum gy[b, o, .]."""
    gx = np.zeros_like(x)
    gw = np.zeros_like(w)
    for t, (dx, dy, dz) in enumerate(TAPS):
        gx += np.einsum("oi,bozyx->bizyx", w[:, :, t], shifted(gy, -dx, -dy, -dz))
        gw[:, :, t] = np.einsum("bozyx,bizyx->oi", gy, shifted(x, dx, dy, dz))
    gb = gy.sum(axis=(0, 2, 3, 4))
    return gx, gw, gb


def mse(pred, target, mask, count):
    """Masked mean-squared error and its gradient."""
    d = (pred - target) * mask
    return float((d * d).sum() / count), 2.0 * d / count


def adam_step(p, g, m, v, lr, b1, b2, eps, step):
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def network_forward(x, layers):
    """layers: list of (w, b); ReLU after every layer but the last.  Returns
    the output and the list of layer inputs (for the backward pass)."""
    acts = [x]
    a = x
    for k, (w, b) in enumerate(layers):
        a = conv_forward(a, w, b, relu=k < len(layers) - 1)
        acts.append(a)
    return a, acts


def network_backward(acts, layers, gy):
    """Gradients of every (w, b) for the output gradient gy."""
    grads = [None] * len(layers)
    g = gy
    for k in range(len(layers) - 1, -1, -1):
        w, _ = layers[k]
        gx, gw, gb = conv_backward(acts[k], w, g)
        grads[k] = (gw, gb)
        if k > 0:
            g = gx * (acts[k] > 0.0)                      # ReLU of the previous layer
    return grads
