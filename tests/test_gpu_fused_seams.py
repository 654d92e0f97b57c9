"""GPU: temporally blocked FGP launches against the one-update-per-launch path.

A fused launch runs K dual updates on a tile with a halo of K + 1 pixels at
the top / left and K at the bottom / right (Algorithm 1's updates need w at
the left / up neighbour for theta and theta at the right / down neighbour for
the gradient).  If a halo were one pixel short anywhere, the pixels next to
the tile seams would differ from the per-update path, which has no seams.
Both paths perform the same FP32 operations in the same order on every pixel,
so the comparison is exact, for every depth K, both outer loops, and shapes
whose extents leave ragged last tiles in both directions.
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import TOL_F32, lib, make_problem, to_dev

pytestmark = pytest.mark.gpu

# One-frame tiles (64 x 128 extended; 32 x 64 for small images at K <= 7) and
# the VTV tiles (32 x 32 for up to 10 frames, 32 x 16 for 16 and 24): several
# tiles per axis, none dividing the extent.
CASES = [("atv", 200, 330, 3), ("atv", 150, 120, 2), ("itv2d", 173, 259, 2), ("vtv", 97, 131, 10),
         ("vtv", 61, 45, 7), ("vtv", 70, 83, 16), ("vtv", 40, 53, 24)]


@pytest.fixture(scope="module")
def pkg():
    return lib()


@pytest.mark.parametrize("algo", ["gap", "admm"])
@pytest.mark.parametrize("tv,nx,ny,B", CASES)
def test_every_depth_bitwise_equal_to_per_update_path(pkg, algo, tv, nx, ny, B):
    case, y = make_problem(nx, ny, B, 90 + nx + B, sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    T, S = 3, 10

    def solve(fuse_k):
        if algo == "gap":
            x, th, _ = pkg.sci_gap_tv(to_dev(y), bits, B, tv, 0.05, T, S, fuse_k=fuse_k)
        else:
            x, th, _, _ = pkg.sci_admm_tv(to_dev(y), bits, B, tv, 0.05, 0.01, T, S, fuse_k=fuse_k)
        return x.cpu().numpy(), th.cpu().numpy()

    x_ref, th_ref = solve(-1)
    # the reference path itself is right: against the FP64 oracle
    ref = (O.gap_tv(y, case.masks, 0.05, T, S, tv) if algo == "gap"
           else O.admm_tv(y, case.masks, 0.05, 0.01, T, S, tv))
    assert np.max(np.abs(th_ref - ref[1])) <= TOL_F32
    for k in (1, 2, 3, 4, 6, 7, 10, 0):
        x, th = solve(k)
        np.testing.assert_array_equal(th, th_ref, err_msg=f"theta, fuse_k={k}")
        np.testing.assert_array_equal(x, x_ref, err_msg=f"x, fuse_k={k}")
