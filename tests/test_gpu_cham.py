"""GPU: the Chambolle TVdenoise box (Algorithm 1, ATV-Cham; ITV2D-Cham and
the ITV3D dual with the norms of Eqs. 29-32) through the C ABI.

The library runs it on the same dual-update kernels as FGP, with every
momentum coefficient zero.  Checks:
- the standalone prox and both outer loops against the FP64 oracle's
  separately written Chambolle box, within max-abs 1e-4;
- every fuse depth bit for bit equal to the per-update path;
- the batched driver bit for bit equal to single solves.
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import TOL_F32, lib, make_problem, maxabs, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    return lib()


@pytest.mark.parametrize("tv", O.TV_TYPES)
@pytest.mark.parametrize("S", [1, 5, 10])
@pytest.mark.parametrize("nx,ny,B", [(1, 1, 1), (37, 70, 3), (64, 96, 8), (9, 33, 32)])
def test_tv_prox_cham(pkg, tv, S, nx, ny, B):
    x = np.random.default_rng(nx + S + B).random((B, nx, ny))
    th = pkg.sci_tv_prox(to_dev(x, torch.float32), tv, 0.05, S, dual="cham")
    assert maxabs(th, O.cham_prox(x.astype(np.float32).astype(np.float64), 0.05, S, tv)) <= TOL_F32


@pytest.mark.parametrize("algo", ["gap", "admm"])
@pytest.mark.parametrize("tv", O.TV_TYPES)
@pytest.mark.parametrize("nx,ny,B", [(37, 70, 3), (130, 150, 10), (9, 33, 32)])
def test_solver_cham(pkg, algo, tv, nx, ny, B):
    case, y = make_problem(nx, ny, B, 60 + B + nx, mask="shifted" if B > 1 else "bernoulli", sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    T, S = 5, 10
    if algo == "gap":
        x, th, _ = pkg.sci_gap_tv(to_dev(y), bits, B, tv, 0.05, T, S, dual="cham")
        xr, thr = O.gap_tv(y, case.masks, 0.05, T, S, tv, dual="cham")
    else:
        x, th, _, _ = pkg.sci_admm_tv(to_dev(y), bits, B, tv, 0.05, 0.01, T, S, dual="cham")
        xr, thr, _ = O.admm_tv(y, case.masks, 0.05, 0.01, T, S, tv, dual="cham")
    assert maxabs(x, xr) <= TOL_F32 and maxabs(th, thr) <= TOL_F32


@pytest.mark.parametrize("tv,nx,ny,B", [("atv", 200, 330, 3), ("itv2d", 173, 259, 2), ("vtv", 97, 131, 10)])
def test_cham_every_depth_bitwise_equal_to_per_update_path(pkg, tv, nx, ny, B):
    case, y = make_problem(nx, ny, B, 5 + nx, sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    ref = None
    for k in (-1, 1, 3, 6, 10, 0):
        x, th, _ = pkg.sci_gap_tv(to_dev(y), bits, B, tv, 0.05, 3, 10, fuse_k=k, dual="cham")
        got = (x.cpu().numpy(), th.cpu().numpy())
        if ref is None:
            ref = got
            continue
        np.testing.assert_array_equal(got[0], ref[0], err_msg=f"x, fuse_k={k}")
        np.testing.assert_array_equal(got[1], ref[1], err_msg=f"theta, fuse_k={k}")


def test_batched_cham_bitwise_equal_to_single_solves(pkg):
    sizes = [(70, 90, 8), (130, 64, 10), (40, 50, 24)]
    ys, bits, Bs, refs = [], [], [], []
    for k, (nx, ny, B) in enumerate(sizes):
        case, y = make_problem(nx, ny, B, 300 + k, sigma=0.01)
        bb = pkg.sci_masks_pack(to_dev(case.masks))
        ys.append(to_dev(y))
        bits.append(bb)
        Bs.append(B)
        x, _, _ = pkg.sci_gap_tv(ys[-1], bb, B, "vtv", 0.05, 4, 5, dual="cham")
        refs.append(x.cpu().numpy())
    batch = pkg.Batch(ys, bits, Bs)
    xs, _ = pkg.sci_gap_tv_batched(batch, "vtv", 0.05, 4, 5, dual="cham")
    for x, r in zip(xs, refs):
        np.testing.assert_array_equal(x.cpu().numpy(), r)
