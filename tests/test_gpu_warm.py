"""GPU: the dual warm start across outer iterations (Algorithm 1 initialises
w once, before its outer loop; nu is reset inside the TVdenoise box).

The temporally blocked solver carries the box's final w (FGP: its last
momentum point; Chambolle box: its w) from one TVdenoise call to the next.
Checks, through the C ABI:
- GAP-TV and ADMM-TV with the FGP and Chambolle boxes against the FP64
  oracle's warm-started loops (``warm_start=True``), max-abs 1e-4;
- every fuse depth bit for bit equal (FP32 storage);
- resuming: T1 + T2 iterations on one workspace equal T bit for bit (the
  carried w stays in the workspace between calls);
- warm start off gives the cold-start result unchanged.
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import TOL_F32, lib, make_problem, maxabs, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    return lib()


def _solve(pkg, algo, y, bits, B, tv, T, S, dual="fgp", **kw):
    if algo == "gap":
        x, th, _ = pkg.sci_gap_tv(y, bits, B, tv, 0.05, T, S, dual=dual, **kw)
        return x, th, None
    x, th, u, _ = pkg.sci_admm_tv(y, bits, B, tv, 0.05, 0.01, T, S, dual=dual, **kw)
    return x, th, u


@pytest.mark.parametrize("algo", ["gap", "admm"])
@pytest.mark.parametrize("dual", ["fgp", "cham"])
@pytest.mark.parametrize("tv", O.TV_TYPES)
@pytest.mark.parametrize("nx,ny,B,S", [(37, 70, 3, 2), (130, 150, 10, 3), (64, 96, 8, 10)])
def test_warm_solver_matches_oracle(pkg, algo, dual, tv, nx, ny, B, S):
    case, y = make_problem(nx, ny, B, 70 + B + nx + S, mask="shifted", sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    T = 6
    x, th, u = _solve(pkg, algo, to_dev(y), bits, B, tv, T, S, dual=dual, warm_start=True)
    if algo == "gap":
        xr, thr = O.gap_tv(y, case.masks, 0.05, T, S, tv, dual=dual, warm_start=True)
    else:
        xr, thr, ur = O.admm_tv(y, case.masks, 0.05, 0.01, T, S, tv, dual=dual, warm_start=True)
        assert maxabs(u, ur) <= TOL_F32
    assert maxabs(x, xr) <= TOL_F32 and maxabs(th, thr) <= TOL_F32
    # the warm start changes the result (else the test would not see a missing carry)
    if algo == "gap":
        xc, _ = O.gap_tv(y, case.masks, 0.05, T, S, tv, dual=dual)
    else:
        xc, _, _ = O.admm_tv(y, case.masks, 0.05, 0.01, T, S, tv, dual=dual)
    assert np.max(np.abs(xc - xr)) > 10 * TOL_F32


@pytest.mark.parametrize("algo", ["gap", "admm"])
@pytest.mark.parametrize("tv,nx,ny,B", [("atv", 200, 330, 3), ("itv2d", 173, 259, 2), ("vtv", 97, 131, 10)])
def test_warm_every_depth_bitwise(pkg, algo, tv, nx, ny, B):
    case, y = make_problem(nx, ny, B, 95 + nx, sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    T, S = 4, 10
    ref = None
    for k in (0, 1, 2, 3, 4, 7, 10):
        x, th, _ = _solve(pkg, algo, to_dev(y), bits, B, tv, T, S, warm_start=True, fuse_k=k)
        got = (x.cpu().numpy(), th.cpu().numpy())
        if ref is None:
            ref = got
            continue
        np.testing.assert_array_equal(got[0], ref[0], err_msg=f"x, fuse_k={k}")
        np.testing.assert_array_equal(got[1], ref[1], err_msg=f"theta, fuse_k={k}")


@pytest.mark.parametrize("algo", ["gap", "admm"])
@pytest.mark.parametrize("T1", [1, 2, 3])
def test_warm_resume_bitwise(pkg, algo, T1):
    """T1 + T2 = T: the second call starts from the theta (and u) the first
    returned and from the w it left in the shared workspace.  T1 odd and even
    both occur, so the carried w's ping-pong parity is covered."""
    B, nx, ny, tv, S, T = 6, 70, 90, "vtv", 3, 5
    case, y = make_problem(nx, ny, B, 123, sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    yd = to_dev(y)
    xf, thf, uf = _solve(pkg, algo, yd, bits, B, tv, T, S, warm_start=True, work=pkg.Workspace(yd.device))
    work = pkg.Workspace(yd.device)
    th = torch.empty((B, nx, ny), dtype=torch.float32, device=yd.device)
    u = torch.empty_like(th) if algo == "admm" else None
    kw = dict(warm_start=True, work=work, theta=th)
    if u is not None:
        kw["u"] = u
    _solve(pkg, algo, yd, bits, B, tv, T1, S, init=True, **kw)
    x2, th2, u2 = _solve(pkg, algo, yd, bits, B, tv, T - T1, S, init=False, **kw)
    np.testing.assert_array_equal(x2.cpu().numpy(), xf.cpu().numpy())
    np.testing.assert_array_equal(th2.cpu().numpy(), thf.cpu().numpy())
    if algo == "admm":
        np.testing.assert_array_equal(u2.cpu().numpy(), uf.cpu().numpy())


@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_warm_off_is_the_cold_solve(pkg, tv):
    B, nx, ny = 8, 64, 80
    case, y = make_problem(nx, ny, B, 7, sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    a = _solve(pkg, "gap", to_dev(y), bits, B, tv, 4, 5)[0].cpu().numpy()
    b = _solve(pkg, "gap", to_dev(y), bits, B, tv, 4, 5, warm_start=False)[0].cpu().numpy()
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_warm_16bit_storage_close_to_fp32(pkg, storage):
    """The carried w is stored in the storage type; the reconstruction stays
    within 0.1 dB of the FP32 warm-started one."""
    B, nx, ny = 10, 128, 128
    case, y = make_problem(nx, ny, B, 31, mask="shifted", sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    x32 = _solve(pkg, "gap", to_dev(y), bits, B, "vtv", 30, 2, warm_start=True)[0].cpu().numpy()
    x16 = _solve(pkg, "gap", to_dev(y), bits, B, "vtv", 30, 2, warm_start=True,
                 storage=storage)[0].cpu().numpy()
    assert abs(O.psnr(x16, case.x_gt) - O.psnr(x32, case.x_gt)) <= 0.1
