"""Pins for the learned-prox network oracle (oracle/lprox_oracle.py).

The convolution is checked against scipy.ndimage.correlate (an independent
implementation), its input gradient by the adjoint identity, and the whole
network's gradients by central finite differences in FP64.
"""
import numpy as np
import pytest
from scipy import ndimage

from oracle import lprox_oracle as L


def test_conv3d_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    a = rng.normal(size=(3, 5, 6, 2))
    w = rng.normal(size=(27, 3, 2))
    b = rng.normal(size=3)
    out = L.conv3d(a, w, b)
    for o in range(3):
        ref = np.full(a.shape[:3], b[o])
        for i in range(2):
            k = np.zeros((3, 3, 3))
            for t, (dz, dy, dx) in enumerate(L.TAPS):
                k[dz + 1, dy + 1, dx + 1] = w[t, o, i]
            ref += ndimage.correlate(a[..., i], k, mode="constant", cval=0.0)
        np.testing.assert_allclose(out[..., o], ref, atol=1e-12)


def test_conv3d_input_grad_is_adjoint():
    rng = np.random.default_rng(1)
    a = rng.normal(size=(4, 3, 5, 3))
    w = rng.normal(size=(27, 2, 3))
    g = rng.normal(size=(4, 3, 5, 2))
    lhs = np.sum(L.conv3d(a, w, np.zeros(2)) * g)
    rhs = np.sum(a * L.conv3d_input_grad(g, w))
    assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs))


def test_network_gradients_match_finite_differences():
    rng = np.random.default_rng(2)
    params = L.init_params(C=4, seed=3)
    params = [(w * 3.0, b + 0.1 * rng.normal(size=b.shape)) for w, b in params]  # avoid a dead net
    x = rng.random((3, 6, 5))
    target = x + 0.1 * rng.normal(size=x.shape)
    loss, grads = L.lprox_loss_and_grads(x, target, params)
    eps = 1e-6
    for k in range(4):
        w, b = params[k]
        for idx in [tuple(rng.integers(0, s) for s in w.shape) for _ in range(6)]:
            wp, wm = w.copy(), w.copy()
            wp[idx] += eps
            wm[idx] -= eps
            pp = [(wp if j == k else pw, pb) for j, (pw, pb) in enumerate(params)]
            pm = [(wm if j == k else pw, pb) for j, (pw, pb) in enumerate(params)]
            num = (L.lprox_loss_and_grads(x, target, pp)[0] - L.lprox_loss_and_grads(x, target, pm)[0]) / (2 * eps)
            assert grads[k][0][idx] == pytest.approx(num, rel=1e-5, abs=1e-9)
        j = int(rng.integers(0, b.shape[0]))
        bp, bm = b.copy(), b.copy()
        bp[j] += eps
        bm[j] -= eps
        pp = [(pw, bp if i == k else pb) for i, (pw, pb) in enumerate(params)]
        pm = [(pw, bm if i == k else pb) for i, (pw, pb) in enumerate(params)]
        num = (L.lprox_loss_and_grads(x, target, pp)[0] - L.lprox_loss_and_grads(x, target, pm)[0]) / (2 * eps)
        assert grads[k][1][j] == pytest.approx(num, rel=1e-5, abs=1e-9)


def test_zero_last_layer_is_identity():
    params = L.init_params(C=4, seed=5)
    w4, b4 = params[3]
    params[3] = (np.zeros_like(w4), np.zeros_like(b4))
    x = np.random.default_rng(6).random((2, 4, 4))
    theta, _ = L.lprox_forward(x, params)
    np.testing.assert_array_equal(theta, x)
