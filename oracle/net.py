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


def energy_loss(pred, target, mask, x):
    """Energy norm of the interior error, the norm in which the basis
    functions' error costs the coarse space: with e = mask (pred - target)
    (zero on the patch boundary, whose values are exact) and relative face
    couplings w = exp(x[:, d]) read from the log-coupling input channels
    (channel d at a cell holds the coupling to its lower neighbour along d),
        E = sum_faces w (e_u - e_v)^2 / count,
    count = the number of interior entries.  Returns (E, dE/dpred)."""
    e = (pred - target) * mask
    count = mask.sum()
    g = np.zeros_like(e)
    E = 0.0
    for d, axis in ((0, 4), (1, 3), (2, 2)):            # x, y, z axes of (B, C, z, y, x)
        w = np.exp(x[:, d:d + 1])                         # (B, 1, S, S, S): coupling to the lower cell
        lo = [slice(None)] * 5; hi = [slice(None)] * 5
        lo[axis] = slice(0, -1); hi[axis] = slice(1, None)
        diff = e[tuple(hi)] - e[tuple(lo)]                # e_u - e_{u - 1} at the upper cell u
        wf = w[tuple(hi)]
        E += float((wf * diff * diff).sum())
        gu = 2.0 * wf * diff
        g[tuple(hi)] += gu
        g[tuple(lo)] -= gu
    return E / count, g * mask / count
