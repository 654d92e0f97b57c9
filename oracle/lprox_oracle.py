"""FP64 oracle for the learned TV prox: a 4-layer 3-D convolutional network.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper has no learned component; its future-work paragraph (Sec. 4)
points at plug-and-play reconstruction.  The network restated here is the
build's stand-in for S FGP updates inside GAP-TV:

  f(x) = conv4(relu(conv3(relu(conv2(relu(conv1(x)))))))
  theta = x + f(x)

conv1: 1 -> C channels, conv2, conv3: C -> C, conv4: C -> 1, all 3x3x3 with
zero "same" padding over (frame, row, column) = (B, nx, ny), i.e. frames are
the depth axis.  Activations are channels-last [B][nx][ny][C].  Weights are
stored as w[tap][c_out][c_in] with tap = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)
for offsets dz, dy, dx in {-1, 0, 1}; layer l computes
  out[z, y, x, o] = b[o] + sum_tap sum_i w[tap, o, i] * in[z + dz, y + dy, x + dx, i]
(a cross-correlation; out-of-range inputs are 0).

Loss: mean squared error between theta and a target, over all voxels.
"""
from __future__ import annotations

import numpy as np

__all__ = ["TAPS", "conv3d", "conv3d_input_grad", "conv3d_weight_grad", "lprox_forward",
           "lprox_loss_and_grads", "init_params"]

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _shift(a, dz, dy, dx):
    """s[z, y, x] = a[z + dz, y + dy, x + dx] (0 outside) for a [D][H][W][C] array."""
    out = np.zeros_like(a)
    D, H, W = a.shape[:3]
    zs, ys, xs = slice(max(0, -dz), min(D, D - dz)), slice(max(0, -dy), min(H, H - dy)), \
        slice(max(0, -dx), min(W, W - dx))
    zt, yt, xt = slice(max(0, dz), min(D, D + dz)), slice(max(0, dy), min(H, H + dy)), \
        slice(max(0, dx), min(W, W + dx))
    out[zs, ys, xs] = a[zt, yt, xt]
    return out


def conv3d(a, w, b):
    """Layer output: a [D][H][W][Ci], w [27][Co][Ci], b [Co] -> [D][H][W][Co]."""
    a = np.asarray(a, np.float64)
    out = np.zeros(a.shape[:3] + (w.shape[1],))
    for t, (dz, dy, dx) in enumerate(TAPS):
        out += _shift(a, dz, dy, dx) @ np.asarray(w[t], np.float64).T
    return out + np.asarray(b, np.float64)


def conv3d_input_grad(g, w):
    """d loss / d input of conv3d given g = d loss / d output ([D][H][W][Co])."""
    g = np.asarray(g, np.float64)
    out = np.zeros(g.shape[:3] + (w.shape[2],))
    for t, (dz, dy, dx) in enumerate(TAPS):
        # output (z, y, x) read input (z + dz, ...): scatter back with the opposite shift
        out += _shift(g, -dz, -dy, -dx) @ np.asarray(w[t], np.float64)
    return out


def conv3d_weight_grad(g, a):
    """d loss / d w [27][Co][Ci] and d loss / d b [Co]."""
    g = np.asarray(g, np.float64)
    a = np.asarray(a, np.float64)
    Co, Ci = g.shape[3], a.shape[3]
    dw = np.zeros((27, Co, Ci))
    for t, (dz, dy, dx) in enumerate(TAPS):
        dw[t] = g.reshape(-1, Co).T @ _shift(a, dz, dy, dx).reshape(-1, Ci)
    return dw, g.reshape(-1, Co).sum(axis=0)


def init_params(C=32, seed=0):
    """He-style random initialisation (the last layer scaled down so f starts near 0)."""
    rng = np.random.default_rng(seed)
    shapes = [(27, C, 1), (27, C, C), (27, C, C), (27, 1, C)]
    params = []
    for k, s in enumerate(shapes):
        fan_in = 27 * s[2]
        w = rng.normal(0.0, np.sqrt(2.0 / fan_in), size=s) * (0.1 if k == 3 else 1.0)
        params.append((w, np.zeros(s[1])))
    return params


def lprox_forward(x, params):
    """theta = x + f(x) for x [D][H][W]; also returns the layer activations."""
    a = np.asarray(x, np.float64)[..., None]
    acts = [a]
    for k, (w, b) in enumerate(params):
        z = conv3d(acts[-1], w, b)
        acts.append(np.maximum(z, 0.0) if k < 3 else z)
    return a[..., 0] + acts[-1][..., 0], acts


def lprox_loss_and_grads(x, target, params):
    """MSE loss and its gradients with respect to every (w, b)."""
    theta, acts = lprox_forward(x, params)
    n = theta.size
    diff = theta - np.asarray(target, np.float64)
    loss = float(np.mean(diff * diff))
    g = (2.0 / n) * diff[..., None]  # d loss / d f
    grads = [None] * 4
    for k in (3, 2, 1, 0):
        w, _ = params[k]
        grads[k] = conv3d_weight_grad(g, acts[k])
        if k > 0:
            g = conv3d_input_grad(g, w) * (acts[k] > 0.0)
    return loss, grads
