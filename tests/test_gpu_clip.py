"""GPU: the ATV-Clip TVdenoise box (Algorithm 1, ATV-Clip) through the C ABI.

The library runs it on the dual-update kernels with the duals scaled by the
threshold lambda, no momentum, step 1/(4 lambda), and direction-specific
theta_h, theta_v in the gradient.  Checks:
- the standalone prox and both outer loops against the FP64 oracle's
  separately written clip_prox (unscaled duals), max-abs 1e-4;
- every fuse depth bit for bit equal to the per-update path;
- the dual warm start with the Clip box against the oracle's;
- ITV2D / VTV with the Clip box, and the batched driver, are refused.
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import TOL_F32, lib, make_problem, maxabs, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    return lib()


@pytest.mark.parametrize("S", [1, 5, 10, 25])
@pytest.mark.parametrize("nx,ny,B", [(1, 1, 1), (37, 70, 3), (64, 96, 8), (200, 150, 2)])
def test_tv_prox_clip(pkg, S, nx, ny, B):
    x = np.random.default_rng(nx + S + B).random((B, nx, ny))
    th = pkg.sci_tv_prox(to_dev(x, torch.float32), "atv", 0.05, S, dual="clip")
    assert maxabs(th, O.clip_prox(x.astype(np.float32).astype(np.float64), 0.05, S)) <= TOL_F32


@pytest.mark.parametrize("algo", ["gap", "admm"])
@pytest.mark.parametrize("nx,ny,B", [(37, 70, 3), (130, 150, 10), (9, 33, 32)])
def test_solver_clip(pkg, algo, nx, ny, B):
    case, y = make_problem(nx, ny, B, 61 + B + nx, mask="shifted" if B > 1 else "bernoulli", sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    T, S = 5, 10
    if algo == "gap":
        x, th, _ = pkg.sci_gap_tv(to_dev(y), bits, B, "atv", 0.05, T, S, dual="clip")
        xr, thr = O.gap_tv(y, case.masks, 0.05, T, S, "atv", dual="clip")
    else:
        x, th, _, _ = pkg.sci_admm_tv(to_dev(y), bits, B, "atv", 0.05, 0.01, T, S, dual="clip")
        xr, thr, _ = O.admm_tv(y, case.masks, 0.05, 0.01, T, S, "atv", dual="clip")
    assert maxabs(x, xr) <= TOL_F32 and maxabs(th, thr) <= TOL_F32


@pytest.mark.parametrize("algo", ["gap", "admm"])
@pytest.mark.parametrize("nx,ny,B", [(200, 330, 3), (150, 120, 2)])
def test_clip_every_depth_bitwise(pkg, algo, nx, ny, B):
    case, y = make_problem(nx, ny, B, 90 + nx + B, sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    T, S = 3, 10

    def solve(k):
        if algo == "gap":
            return pkg.sci_gap_tv(to_dev(y), bits, B, "atv", 0.05, T, S, fuse_k=k, dual="clip")[0].cpu().numpy()
        return pkg.sci_admm_tv(to_dev(y), bits, B, "atv", 0.05, 0.01, T, S, fuse_k=k,
                               dual="clip")[0].cpu().numpy()

    ref = solve(-1)
    xr = (O.gap_tv(y, case.masks, 0.05, T, S, "atv", dual="clip")[0] if algo == "gap"
          else O.admm_tv(y, case.masks, 0.05, 0.01, T, S, "atv", dual="clip")[0])
    assert np.max(np.abs(ref - xr)) <= TOL_F32
    for k in (1, 2, 3, 4, 7, 10, 0):
        np.testing.assert_array_equal(solve(k), ref, err_msg=f"fuse_k={k}")


def test_clip_warm_start(pkg):
    B, nx, ny, T, S = 6, 90, 70, 6, 2
    case, y = make_problem(nx, ny, B, 17, mask="shifted", sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    x, _, _ = pkg.sci_gap_tv(to_dev(y), bits, B, "atv", 0.05, T, S, dual="clip", warm_start=True)
    xr, _ = O.gap_tv(y, case.masks, 0.05, T, S, "atv", dual="clip", warm_start=True)
    assert maxabs(x, xr) <= TOL_F32


def test_clip_refusals(pkg):
    B, nx, ny = 4, 32, 32
    case, y = make_problem(nx, ny, B, 3)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    for tv in ("itv2d", "vtv"):
        with pytest.raises(pkg.SciError):
            pkg.sci_gap_tv(to_dev(y), bits, B, tv, 0.05, 2, 3, dual="clip")
        with pytest.raises(pkg.SciError):
            pkg.sci_tv_prox(to_dev(np.zeros((B, nx, ny), np.float32)), tv, 0.05, 3, dual="clip")
    batch = pkg.Batch([to_dev(y)], [bits], [B])
    with pytest.raises(pkg.SciError):
        pkg.sci_gap_tv_batched(batch, "atv", 0.05, 2, 3, dual="clip")
