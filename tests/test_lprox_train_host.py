"""CPU: the learned-prox trainer's host logic, with a stand-in network.

init_params lays the four layers out as the library expects (weights
[27][out][in] then biases, per layer), with He-scaled weights, zero biases
and the output layer at a tenth of its scale.  train runs epochs x
floor(n / batch) Adam steps in a seeded order, with a cosine learning-rate
decay from lr towards 0, floored at lr * 1e-3, and reports the mean loss per
voxel for each epoch; fewer pairs than one batch is an error.
"""
import math

import numpy as np
import pytest
import torch

from paper_2005_08028_gb300 import lprox_train as LT
from paper_2005_08028_gb300 import sci as S


@pytest.fixture(scope="module")
def lib():
    from paper_2005_08028_gb300 import build as b
    return S.load(b.build())


def _layers(flat):
    C, out = 32, []
    off = 0
    for co, ci in [(C, 1), (C, C), (C, C), (1, C)]:
        w = flat[off:off + 27 * co * ci].reshape(27, co, ci)
        off += 27 * co * ci
        b = flat[off:off + co]
        off += co
        out.append((w, b, ci))
    assert off == flat.size
    return out


def test_init_params_layout_and_scales(lib):
    flat = LT.init_params(seed=3, device="cpu").numpy().astype(np.float64)
    assert flat.size == S.LearnedProx.param_count()
    layers = _layers(flat)
    for k, (w, b, ci) in enumerate(layers):
        assert np.all(b == 0.0)
        want = math.sqrt(2.0 / (27 * ci)) * (0.1 if k == 3 else 1.0)
        assert w.std() == pytest.approx(want, rel=0.25 if k == 3 else 0.05)
    # seeded: the same seed gives the same weights, another seed others
    assert np.array_equal(flat, LT.init_params(seed=3, device="cpu").numpy())
    assert not np.array_equal(flat, LT.init_params(seed=4, device="cpu").numpy())


class FakeNet:
    """Records the learning rates and batches train() hands to train_step."""

    def __init__(self):
        self.lrs, self.batches = [], []

    def train_step(self, x, y, lr):
        self.lrs.append(lr)
        self.batches.append(x[:, 0, 0, 0].clone())
        return (x - y).pow(2).sum()  # summed squared error, as the library returns


def test_train_schedule_order_and_loss_normalisation():
    n, batch, epochs, lr = 70, 16, 3, 1e-3
    X = torch.arange(n, dtype=torch.float32).reshape(n, 1, 1, 1).expand(n, 2, 3, 4).contiguous()
    Y = X - 0.5  # every voxel off by 0.5: mean squared error per voxel 0.25
    net = FakeNet()
    hist = LT.train(net, X, Y, epochs=epochs, batch=batch, lr=lr, seed=5)
    steps = epochs * (n // batch)
    assert len(net.lrs) == steps and len(hist) == epochs
    want = [max(lr * 0.5 * (1 + math.cos(math.pi * k / steps)), lr * 1e-3) for k in range(steps)]
    assert net.lrs == pytest.approx(want)
    assert net.lrs[0] == pytest.approx(lr) and all(a >= b for a, b in zip(net.lrs, net.lrs[1:]))
    assert hist == pytest.approx([0.25] * epochs)
    # each epoch visits distinct samples; the order is seeded
    for e in range(epochs):
        seen = torch.cat(net.batches[e * (n // batch):(e + 1) * (n // batch)])
        assert len(set(seen.tolist())) == seen.numel() == (n // batch) * batch
    again = FakeNet()
    LT.train(again, X, Y, epochs=epochs, batch=batch, lr=lr, seed=5)
    assert all(torch.equal(a, b) for a, b in zip(net.batches, again.batches))


def test_train_needs_at_least_one_batch():
    X = torch.zeros(5, 1, 2, 2)
    net = FakeNet()
    with pytest.raises(ValueError):
        LT.train(net, X, X, epochs=2, batch=8)
    with pytest.raises(ValueError):
        LT.train(net, X, X, epochs=2, batch=0)
    assert net.lrs == []
    assert LT.train(net, X, X, epochs=1, batch=5) == [0.0] and len(net.lrs) == 1
