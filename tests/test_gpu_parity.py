"""GPU parity: libsci (through its C ABI) against the FP64 oracle on seeded inputs.

Tolerance: FP32 results within max-abs 1e-4 per voxel of the FP64 oracle.
Shapes span several 32x8 pixel tiles with ragged tails, plus degenerate
1-pixel-wide cases and B = 1 and B = 32.
"""
import numpy as np
import pytest

import oracle as O
import sci_synth as ss
from gpu_helpers import TOL_F32, lib, make_problem, maxabs, to_dev, torch

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (1, 70, 2), (70, 1, 2), (37, 70, 3), (64, 96, 8), (9, 33, 32)]


@pytest.fixture(scope="module")
def pkg():
    return lib()


@pytest.mark.parametrize("nx,ny,B", SHAPES)
def test_pack_forward_adjoint(pkg, nx, ny, B):
    case, y = make_problem(nx, ny, B, 11 + nx + B)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    np.testing.assert_array_equal(bits.cpu().numpy().view(np.uint32), ss.pack_mask_bits(case.masks))
    yg = pkg.sci_forward(to_dev(case.x_gt, torch.float32), bits)
    np.testing.assert_allclose(yg.cpu().numpy(), O.forward(case.x_gt.astype(np.float32), case.masks),
                               atol=1e-5 * B, rtol=0)
    xg = pkg.sci_adjoint(to_dev(y), bits, B)
    np.testing.assert_array_equal(xg.cpu().numpy(), O.adjoint(y, case.masks).astype(np.float32))


def test_pack_rejects_non_binary(pkg):
    m = np.zeros((2, 4, 4), np.uint8)
    m[1, 2, 3] = 2
    with pytest.raises(ValueError):
        pkg.sci_masks_pack(to_dev(m))


@pytest.mark.parametrize("nx,ny,B", SHAPES)
@pytest.mark.parametrize("rho", [0.0, 0.01])
def test_project(pkg, nx, ny, B, rho):
    case, y = make_problem(nx, ny, B, 5 + nx, sigma=0.01)
    m = case.masks.copy()
    m[:, 0, 0] = 0  # force an R = 0 pixel
    rng = np.random.default_rng(nx * ny + B)
    theta = rng.random((B, nx, ny)).astype(np.float32)
    u = (0.1 * rng.standard_normal((B, nx, ny))).astype(np.float32)
    bits = pkg.sci_masks_pack(to_dev(m))
    if rho == 0.0:
        xg = pkg.sci_project(to_dev(theta), to_dev(y), bits)
        ref = O.gap_project(theta, y, m)
    else:
        xg = pkg.sci_project(to_dev(theta), to_dev(y), bits, rho=rho, u=to_dev(u))
        ref = O.admm_xupdate(theta, u, y, m, rho)
    assert maxabs(xg, ref) <= 1e-5


@pytest.mark.parametrize("tv", O.TV_TYPES)
@pytest.mark.parametrize("S", [1, 2, 5, 10])
@pytest.mark.parametrize("nx,ny,B", [(1, 1, 1), (1, 40, 2), (37, 70, 3), (64, 96, 8)])
def test_tv_prox(pkg, tv, S, nx, ny, B):
    x = np.random.default_rng(S * 100 + nx).random((B, nx, ny)).astype(np.float32)
    th = pkg.sci_tv_prox(to_dev(x), tv, 0.05, S)
    assert maxabs(th, O.fgp_prox(x, 0.05, S, tv)) <= 1e-5


@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_tv_prox_constant_frames_fixed(pkg, tv):
    x = np.stack([np.full((20, 45), v, np.float32) for v in (0.25, 0.5, 0.75)])
    th = pkg.sci_tv_prox(to_dev(x), tv, 0.05, 7)
    np.testing.assert_array_equal(th.cpu().numpy(), x)


@pytest.mark.parametrize("algo", ["gap", "admm"])
@pytest.mark.parametrize("tv", O.TV_TYPES)
@pytest.mark.parametrize("nx,ny,B", [(1, 1, 1), (37, 70, 3), (64, 96, 8), (9, 33, 32)])
def test_solver_small(pkg, algo, tv, nx, ny, B):
    case, y = make_problem(nx, ny, B, 21 + B, mask="shifted" if B > 1 else "bernoulli", sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    T, S = 6, 4
    if algo == "gap":
        x, th, _ = pkg.sci_gap_tv(to_dev(y), bits, B, tv, 0.05, T, S)
        xr, thr = O.gap_tv(y, case.masks, 0.05, T, S, tv)
        assert maxabs(x, xr) <= TOL_F32 and maxabs(th, thr) <= TOL_F32
    else:
        x, th, u, _ = pkg.sci_admm_tv(to_dev(y), bits, B, tv, 0.05, 0.01, T, S)
        xr, thr, ur = O.admm_tv(y, case.masks, 0.05, 0.01, T, S, tv)
        assert maxabs(x, xr) <= TOL_F32 and maxabs(th, thr) <= TOL_F32 and maxabs(u, ur) <= TOL_F32


@pytest.mark.parametrize("fuse_k", [-1, 1, 3, 0, 7])
@pytest.mark.parametrize("algo", ["gap", "admm"])
@pytest.mark.parametrize("tv,nx,ny,B", [("atv", 150, 300, 3), ("itv2d", 70, 130, 2), ("vtv", 150, 100, 10),
                                        ("vtv", 45, 70, 7), ("vtv", 40, 50, 12), ("vtv", 20, 30, 20)])
def test_solver_fused_depths(pkg, fuse_k, algo, tv, nx, ny, B):
    """Every temporal-blocking depth (and the per-update path, fuse_k = -1)
    matches the oracle on sizes spanning several tiles with ragged tails."""
    case, y = make_problem(nx, ny, B, 7 * B + nx, sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    T, S = 3, 8
    if algo == "gap":
        x, th, _ = pkg.sci_gap_tv(to_dev(y), bits, B, tv, 0.05, T, S, fuse_k=fuse_k)
        xr, thr = O.gap_tv(y, case.masks, 0.05, T, S, tv)
    else:
        x, th, _, _ = pkg.sci_admm_tv(to_dev(y), bits, B, tv, 0.05, 0.01, T, S, fuse_k=fuse_k)
        xr, thr, _ = O.admm_tv(y, case.masks, 0.05, 0.01, T, S, tv)
    assert maxabs(x, xr) <= TOL_F32 and maxabs(th, thr) <= TOL_F32


@pytest.mark.parametrize("tv", O.TV_TYPES)
@pytest.mark.parametrize("S", [1, 10, 25])
def test_tv_prox_large_tiles(pkg, tv, S):
    x = np.random.default_rng(S).random((10, 300, 260)).astype(np.float32)
    th = pkg.sci_tv_prox(to_dev(x), tv, 0.05, S)
    assert maxabs(th, O.fgp_prox(x, 0.05, S, tv)) <= 1e-5


def test_gap_atv_256x256x8_full(pkg):
    """The 256x256x8 workload at its stated iterations (T = 50, S = 5, ATV, lambda = 0.05)."""
    cfg = ss.CONFIGS["gap_atv_256x256x8"]
    case, y = make_problem(cfg["nx"], cfg["ny"], cfg["B"], cfg["seed"], mask=cfg["mask"],
                           sigma=cfg["sigma"])
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    x, th, _ = pkg.sci_gap_tv(to_dev(y), bits, cfg["B"], "atv", cfg["lam"], cfg["outer"], cfg["inner"])
    xr, thr = O.gap_tv(y, case.masks, cfg["lam"], cfg["outer"], cfg["inner"], "atv")
    assert maxabs(x, xr) <= TOL_F32 and maxabs(th, thr) <= TOL_F32
    dpsnr = abs(O.psnr(x.cpu().numpy(), case.x_gt) - O.psnr(xr, case.x_gt))
    assert dpsnr <= 0.05


@pytest.mark.parametrize("algo", ["gap", "admm"])
def test_resume_and_graph_bitwise(pkg, algo):
    case, y = make_problem(48, 80, 5, 9, sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    yd = to_dev(y)
    if algo == "gap":
        x_full, th_full, _ = pkg.sci_gap_tv(yd, bits, 5, "vtv", 0.05, 7, 3)
        x_eager, th_eager, _ = pkg.sci_gap_tv(yd, bits, 5, "vtv", 0.05, 7, 3, use_graph=False)
        _, th1, _ = pkg.sci_gap_tv(yd, bits, 5, "vtv", 0.05, 4, 3)
        x2, th2, _ = pkg.sci_gap_tv(yd, bits, 5, "vtv", 0.05, 3, 3, theta=th1.clone())
    else:
        x_full, th_full, _, _ = pkg.sci_admm_tv(yd, bits, 5, "vtv", 0.05, 0.01, 7, 3)
        x_eager, th_eager, _, _ = pkg.sci_admm_tv(yd, bits, 5, "vtv", 0.05, 0.01, 7, 3, use_graph=False)
        _, th1, u1, _ = pkg.sci_admm_tv(yd, bits, 5, "vtv", 0.05, 0.01, 4, 3)
        x2, th2, _, _ = pkg.sci_admm_tv(yd, bits, 5, "vtv", 0.05, 0.01, 3, 3, theta=th1.clone(),
                                        u=u1.clone())
    assert torch.equal(x_full, x_eager) and torch.equal(th_full, th_eager)
    assert torch.equal(x2, x_full) and torch.equal(th2, th_full)


def test_residual_history_and_reductions(pkg):
    case, y = make_problem(40, 64, 6, 13, sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    x, th, resid = pkg.sci_gap_tv(to_dev(y), bits, 6, "itv2d", 0.05, 6, 3, resid_every=2)
    refs = []
    for T in (2, 4, 6):
        _, thr = O.gap_tv(y, case.masks, 0.05, T, 3, "itv2d")
        refs.append(O.residual_sq(thr, y, case.masks))
    np.testing.assert_allclose(resid.cpu().numpy(), refs, rtol=1e-4)
    r = pkg.sci_residual_f64(th, to_dev(y), bits)
    assert float(r.item()) == pytest.approx(refs[-1], rel=1e-4)
    a = np.random.default_rng(1).random(100003).astype(np.float32)
    b = np.random.default_rng(2).random(100003).astype(np.float32)
    s = pkg.sci_sqdiff_f64(to_dev(a), to_dev(b))
    assert float(s.item()) == pytest.approx(float(np.sum((a.astype(np.float64) - b) ** 2)), rel=1e-12)


def test_outputs_feasible_on_covered_pixels(pkg):
    case, y = make_problem(64, 64, 8, 31, sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    x, _, _ = pkg.sci_gap_tv(to_dev(y), bits, 8, "atv", 0.05, 10, 5)
    R = case.masks.sum(0)
    yy = O.forward(x.cpu().numpy(), case.masks)
    np.testing.assert_allclose(yy[R > 0], y[R > 0], atol=2e-5)


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_reduced_precision_storage(pkg, storage):
    """16-bit storage with FP32 math: PSNR within 0.1 dB of the FP64 oracle."""
    case, y = make_problem(128, 128, 8, 41)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    x, th, _ = pkg.sci_gap_tv(to_dev(y), bits, 8, "itv2d", 0.05, 20, 5, storage=storage)
    xr, _ = O.gap_tv(y, case.masks, 0.05, 20, 5, "itv2d")
    d = abs(O.psnr(x.cpu().numpy(), case.x_gt) - O.psnr(xr, case.x_gt))
    assert np.isfinite(x.cpu().numpy()).all() and d <= 0.1
    x2, th2, u2, _ = pkg.sci_admm_tv(to_dev(y), bits, 8, "vtv", 0.05, 0.01, 20, 5, storage=storage)
    xr2, _, _ = O.admm_tv(y, case.masks, 0.05, 0.01, 20, 5, "vtv")
    d2 = abs(O.psnr(x2.cpu().numpy(), case.x_gt) - O.psnr(xr2, case.x_gt))
    assert d2 <= 0.1


@pytest.mark.parametrize("algo", ["gap", "admm"])
@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_512x512x10_full_size_short_run(pkg, algo, tv):
    """Full 512x512x10 size (shifted mask, sigma = 0.01) with the solver's own
    launch configuration, for T = 2 outer x S = 10 inner iterations."""
    cfg = ss.CONFIGS["sci_512x512x10"]
    case, y = make_problem(cfg["nx"], cfg["ny"], cfg["B"], cfg["seed"], mask=cfg["mask"],
                           sigma=cfg["sigma"])
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    T, S = 2, cfg["inner"]
    if algo == "gap":
        x, th, _ = pkg.sci_gap_tv(to_dev(y), bits, cfg["B"], tv, cfg["lam"], T, S)
        xr, thr = O.gap_tv(y, case.masks, cfg["lam"], T, S, tv)
    else:
        x, th, _, _ = pkg.sci_admm_tv(to_dev(y), bits, cfg["B"], tv, cfg["lam"], cfg["rho"], T, S)
        xr, thr, _ = O.admm_tv(y, case.masks, cfg["lam"], cfg["rho"], T, S, tv)
    assert maxabs(x, xr) <= TOL_F32 and maxabs(th, thr) <= TOL_F32
