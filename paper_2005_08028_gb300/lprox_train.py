"""Training data and training loop for the learned TV prox.

Pairs (x, FGP_S(x)) come from the plain method itself: GAP-TV runs on seeded
synthetic measurements are stopped at random outer iterations t, the
projection x = P(theta^(t)) is the network input and S FGP dual updates of
it are the target; 64 x 64 patches (all frames) are cut from both.  Every
step runs in libsci (sci_gap_tv, sci_project, sci_tv_prox for the data;
sci_lprox_train_step for training); this module only orchestrates.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import sci as S


def make_pairs(n_patches: int, seed: int, *, size=(256, 256, 8), patch=64, tv="vtv", lam=0.05, inner=10,
               t_range=(1, 50), sigma=0.01, device="cuda"):
    """n_patches (input, target) pairs, each float32 [B][patch][patch] on the device."""
    import sci_synth as ss
    nx, ny, B = size
    dev = torch.device(device)
    rng = np.random.default_rng(seed)
    xs, ts = [], []
    per_frame = (nx // patch) * (ny // patch)
    vid = 0
    while len(xs) * per_frame < n_patches:
        case = ss.make_case(nx, ny, B, seed * 100003 + vid, sigma=sigma)
        vid += 1
        bits = S.sci_masks_pack(torch.from_numpy(case.masks).to(dev))
        y = S.sci_forward(torch.from_numpy(case.x_gt.astype(np.float32)).to(dev), bits) + \
            torch.from_numpy(case.noise.astype(np.float32)).to(dev)
        stops = sorted(set(int(v) for v in rng.integers(t_range[0], t_range[1] + 1, size=3)))
        theta, done = None, 0
        for t in stops:
            if theta is None:
                _, theta, _ = S.sci_gap_tv(y, bits, B, tv, lam, t, inner)
            else:
                _, theta, _ = S.sci_gap_tv(y, bits, B, tv, lam, t - done, inner, theta=theta)
            done = t
            x = S.sci_project(theta, y, bits)
            target = S.sci_tv_prox(x, tv, lam, inner)
            xs.append(x)
            ts.append(target)
    X = torch.stack(xs)  # [n][B][nx][ny]
    T = torch.stack(ts)
    # cut patches
    Xp = X.unfold(2, patch, patch).unfold(3, patch, patch)  # [n][B][px][py][patch][patch]
    Tp = T.unfold(2, patch, patch).unfold(3, patch, patch)
    Xp = Xp.permute(0, 2, 3, 1, 4, 5).reshape(-1, B, patch, patch)
    Tp = Tp.permute(0, 2, 3, 1, 4, 5).reshape(-1, B, patch, patch)
    perm = torch.from_numpy(rng.permutation(Xp.shape[0])[:n_patches]).to(dev)
    return Xp[perm].contiguous(), Tp[perm].contiguous()


def init_params(seed: int = 0, device="cuda") -> torch.Tensor:
    """He-style initialisation; the last layer starts at 0.1x so f(x) starts near 0."""
    rng = np.random.default_rng(seed)
    C = 32
    parts = []
    for k, (co, ci) in enumerate([(C, 1), (C, C), (C, C), (1, C)]):
        w = rng.normal(0.0, math.sqrt(2.0 / (27 * ci)), size=(27, co, ci)) * (0.1 if k == 3 else 1.0)
        parts += [w.reshape(-1), np.zeros(co)]
    flat = np.concatenate(parts).astype(np.float32)
    assert flat.size == S.LearnedProx.param_count()
    return torch.from_numpy(flat).to(device)


def train(net: "S.LearnedProx", X: torch.Tensor, Y: torch.Tensor, *, epochs=8, batch=32, lr=1e-3, seed=0):
    """Adam with cosine learning-rate decay; returns the mean loss per epoch.

    A peak rate of 1e-3 trains reliably; 3e-3 and above left every ReLU dead
    (the network collapsed to f = 0) in our runs."""
    n = X.shape[0]
    if batch < 1 or n < batch:
        raise ValueError(f"need at least one batch of pairs: {n} pairs, batch {batch}")
    steps = epochs * (n // batch)
    g = torch.Generator(device="cpu").manual_seed(seed)
    hist, k = [], 0
    for _ in range(epochs):
        order = torch.randperm(n, generator=g)
        tot, m = 0.0, 0
        for i in range(0, n - batch + 1, batch):
            idx = order[i:i + batch].to(X.device)
            cur = lr * 0.5 * (1.0 + math.cos(math.pi * k / steps))
            loss = net.train_step(X[idx].contiguous(), Y[idx].contiguous(), max(cur, lr * 1e-3))
            tot += float(loss.item()) / (batch * X[0].numel())
            m += 1
            k += 1
        hist.append(tot / max(m, 1))
    return hist
