"""GPU: FISTA-TV (Sec. 2.2, FISTA steps) through the C ABI against the FP64 oracle.

The library forms FISTA's gradient step with the GAP residual kernels, the
1/R field replaced by the constant 1/L (L = max R, taken on the device).  It
runs TVdenoise on the same fused kernels, then one momentum kernel per
iteration.  Checks:
- parity with the oracle within max-abs 1e-4, on the fused and per-update
  paths, for both TVdenoise boxes;
- every fuse depth bit for bit equal to the per-update path;
- FP16 storage within 0.1 dB PSNR of FP32;
- the recorded residuals are ||y - Phi x^(t)||^2.
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import TOL_F32, lib, make_problem, maxabs, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    return lib()


@pytest.mark.parametrize("dual", ["fgp", "cham"])
@pytest.mark.parametrize("tv", O.TV_TYPES)
@pytest.mark.parametrize("nx,ny,B", [(1, 1, 1), (37, 70, 3), (130, 150, 10), (9, 33, 32)])
def test_fista_matches_oracle(pkg, dual, tv, nx, ny, B):
    case, y = make_problem(nx, ny, B, 80 + nx + B, mask="shifted" if B > 1 else "bernoulli", sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    T, S = 6, 8
    x, th, _ = pkg.sci_fista_tv(to_dev(y), bits, B, tv, 0.05, T, S, dual=dual)
    xr, _ = O.fista_tv(y, case.masks, 0.05, T, S, tv, dual=dual)
    assert maxabs(x, xr) <= TOL_F32
    assert torch.equal(x, th)  # both hold x^(T)


@pytest.mark.parametrize("tv,nx,ny,B", [("atv", 200, 330, 3), ("itv2d", 173, 259, 2), ("vtv", 97, 131, 10)])
def test_fista_every_depth_bitwise_equal_to_per_update_path(pkg, tv, nx, ny, B):
    case, y = make_problem(nx, ny, B, 9 + nx, sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    ref = None
    for k in (-1, 1, 4, 10, 0):
        x, _, _ = pkg.sci_fista_tv(to_dev(y), bits, B, tv, 0.05, 4, 10, fuse_k=k)
        got = x.cpu().numpy()
        if ref is None:
            ref = got
        else:
            np.testing.assert_array_equal(got, ref, err_msg=f"fuse_k={k}")


def test_fista_f16_storage_close_to_f32(pkg):
    case, y = make_problem(256, 256, 8, 17, sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    gt = to_dev(case.x_gt.astype(np.float32))
    ps = {}
    for st in ("f32", "f16"):
        x, _, _ = pkg.sci_fista_tv(to_dev(y), bits, 8, "vtv", 0.05, 40, 10, storage=st)
        mse = float(pkg.sci_sqdiff_f64(x, gt).item()) / x.numel()
        ps[st] = 10 * np.log10(1.0 / mse)
    assert abs(ps["f16"] - ps["f32"]) <= 0.1, ps


def test_fista_residual_history(pkg):
    """resid[t-1] is ||y - Phi x^(t)||^2 of the solve's own x^(t): a T = t solve
    runs the same arithmetic up to iteration t, and its x is checked here in
    FP64 against the recorded value."""
    case, y = make_problem(40, 56, 6, 23, sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    T = 6
    _, _, resid = pkg.sci_fista_tv(to_dev(y), bits, 6, "itv2d", 0.05, T, 5, resid_every=1)
    got = resid.cpu().numpy()
    for t in range(1, T + 1):
        xt, _, _ = pkg.sci_fista_tv(to_dev(y), bits, 6, "itv2d", 0.05, t, 5)
        ref = O.residual_sq(xt.cpu().numpy().astype(np.float64), y.astype(np.float32), case.masks)
        assert abs(got[t - 1] - ref) <= 1e-6 * ref, (t, got[t - 1], ref)


def test_graph_cache_keeps_solvers_apart(pkg):
    """The library replays a cached CUDA graph when a solve's arguments repeat.
    GAP-FGP, FISTA-FGP and GAP-Chambolle on the same buffers and workspace
    must each give what a fresh call gives, also when interleaved."""
    case, y = make_problem(60, 70, 8, 41, sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    yd = to_dev(y)
    th = torch.empty((8, 60, 70), device=yd.device)
    xo = torch.empty_like(th)
    work = pkg.Workspace(yd.device)
    runs = [("gap", "fgp"), ("fista", "fgp"), ("gap", "cham"), ("gap", "fgp"), ("fista", "fgp")]
    fresh = {}
    for algo, dual in set(runs):
        f = pkg.sci_fista_tv if algo == "fista" else pkg.sci_gap_tv
        x, _, _ = f(yd, bits, 8, "vtv", 0.05, 5, 6, dual=dual, use_graph=False)
        fresh[(algo, dual)] = x.cpu().numpy()
    for algo, dual in runs:
        f = pkg.sci_fista_tv if algo == "fista" else pkg.sci_gap_tv
        f(yd, bits, 8, "vtv", 0.05, 5, 6, dual=dual, theta=th, x_out=xo, init=True, work=work)
        np.testing.assert_array_equal(xo.cpu().numpy(), fresh[(algo, dual)], err_msg=f"{algo}/{dual}")


def test_fista_zero_iterations_returns_the_start(pkg):
    case, y = make_problem(20, 30, 4, 43)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    x, th, _ = pkg.sci_fista_tv(to_dev(y), bits, 4, "atv", 0.05, 0, 5)
    ref = O.adjoint(y.astype(np.float32).astype(np.float64), case.masks)
    assert maxabs(x, ref) <= 1e-6 and maxabs(th, ref) <= 1e-6
