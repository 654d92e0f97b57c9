"""GPU test of sci_tv_prox_noalloc, the FGP prox whose scratch lives in a fixed
array inside the library (for callers that cannot allocate device memory).

It must give the same result as sci_tv_prox, which takes caller-provided
scratch, on two calls in a row (the second reuses the array the first one
left behind), and refuse sizes beyond its fixed capacity.  This file is named
to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

from gpu_helpers import lib, to_dev, torch

pytestmark = pytest.mark.gpu

TOL = 1e-5  # the prox parity tolerance used by the other GPU tests


@pytest.fixture(scope="module")
def handles():
    pkg = lib()
    h = pkg.sci.load()
    h.sci_tv_prox_noalloc.restype = C.c_int
    h.sci_tv_prox_noalloc.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_float, C.c_int,
                                      C.c_void_p, C.c_void_p]
    h.sci_tv_prox_noalloc_max_voxels.restype = C.c_longlong
    h.sci_tv_prox_noalloc_max_voxels.argtypes = []
    return pkg, h


def _noalloc(h, x, tv, lam, S):
    B, nx, ny = x.shape
    theta = torch.empty_like(x)
    stream = C.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)
    st = h.sci_tv_prox_noalloc(C.c_void_p(x.data_ptr()), nx, ny, B, {"atv": 0, "itv2d": 1, "vtv": 2}[tv],
                               lam, S, C.c_void_p(theta.data_ptr()), stream)
    assert st == 0, st
    return theta


@pytest.mark.parametrize("tv", ["atv", "itv2d", "vtv"])
def test_noalloc_matches_workspace_prox_twice(handles, tv):
    pkg, h = handles
    rng = np.random.default_rng(2024)
    # two calls in a row with different inputs and sizes; the second runs on
    # whatever the first one left in the shared array
    cases = [(rng.random((8, 512, 512)).astype(np.float32), 10),
             (rng.random((3, 37, 70)).astype(np.float32), 5)]
    for x_h, S in cases:
        x = to_dev(x_h)
        got = _noalloc(h, x, tv, 0.05, S)
        want = pkg.sci_tv_prox(x, tv, 0.05, S)
        torch.cuda.synchronize()
        assert float((got - want).abs().max()) <= TOL


def test_noalloc_rejects_oversized(handles):
    _, h = handles
    cap = h.sci_tv_prox_noalloc_max_voxels()
    assert cap == 512 * 512 * 8
    x = torch.zeros(4, device="cuda")  # never read: the size check comes first
    y = torch.zeros(4, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = h.sci_tv_prox_noalloc(C.c_void_p(x.data_ptr()), 512, 512, 9, 0, 0.05, 5, C.c_void_p(y.data_ptr()),
                               stream)
    assert st == 2  # SCI_ERR_SHAPE
