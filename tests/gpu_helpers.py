"""Shared helpers for the GPU parity tests (inputs come from sci_synth + oracle only)."""
import numpy as np
import pytest

import oracle as O
import sci_synth as ss

torch = pytest.importorskip("torch")

TOL_F32 = 1e-4  # max-abs per voxel, FP32 path vs FP64 oracle


def dev():
    return torch.device("cuda:0")


def lib():
    from paper_2005_08028_gb300 import build as b
    b.build()
    import paper_2005_08028_gb300 as pkg
    pkg.sci.load()
    return pkg


def make_problem(nx, ny, B, seed, mask="bernoulli", sigma=0.0):
    """Case plus its FP32 measurement y (formed by the oracle's forward model)."""
    case = ss.make_case(nx, ny, B, seed, mask=mask, sigma=sigma)
    y32 = (O.forward(case.x_gt, case.masks) + case.noise).astype(np.float32)
    return case, y32


def to_dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a)).to(dev())
    return t if dtype is None else t.to(dtype)


def maxabs(gpu_t, ref):
    return float(np.abs(gpu_t.detach().cpu().numpy().astype(np.float64) - ref).max())
