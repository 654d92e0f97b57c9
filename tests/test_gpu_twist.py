"""GPU: TwIST-TV (Sec. 2.2, TwIST steps) through the C ABI.

The library runs TwIST's z-step with FISTA's residual kernels (1/L field,
L = max R), TVdenoise on the temporally blocked kernels (or the per-update
ones), alpha and beta formed on the device from the mask counts, and the
two-step combination in one elementwise kernel.  Checks:
- x^(T) against the FP64 oracle's twist_tv, max-abs 1e-4, for the three TV
  forms and both TVdenoise boxes;
- every fuse depth, and the per-update path, bit for bit equal (FP32);
- the residual history ||y - Phi x^(t)||^2 against the oracle's iterates;
- 16-bit storage within 0.1 dB of FP32.
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import TOL_F32, lib, make_problem, maxabs, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    return lib()


@pytest.mark.parametrize("dual", ["fgp", "cham"])
@pytest.mark.parametrize("tv", O.TV_TYPES)
@pytest.mark.parametrize("nx,ny,B", [(37, 70, 3), (130, 150, 10), (9, 33, 32)])
def test_twist_matches_oracle(pkg, dual, tv, nx, ny, B):
    case, y = make_problem(nx, ny, B, 80 + nx + B, mask="shifted" if B > 1 else "bernoulli", sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    T, S = 6, 5
    x, th, _ = pkg.sci_twist_tv(to_dev(y), bits, B, tv, 0.05, T, S, dual=dual)
    xr, _ = O.twist_tv(y, case.masks, 0.05, T, S, tv, dual=dual)
    assert maxabs(x, xr) <= TOL_F32
    np.testing.assert_array_equal(x.cpu().numpy(), th.cpu().numpy())


@pytest.mark.parametrize("tv,nx,ny,B", [("atv", 200, 330, 3), ("itv2d", 173, 259, 2), ("vtv", 97, 131, 10)])
def test_twist_every_depth_bitwise(pkg, tv, nx, ny, B):
    case, y = make_problem(nx, ny, B, 33 + nx, sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    T, S = 4, 10
    ref = pkg.sci_twist_tv(to_dev(y), bits, B, tv, 0.05, T, S, fuse_k=-1)[0].cpu().numpy()
    xr, _ = O.twist_tv(y, case.masks, 0.05, T, S, tv)
    assert np.max(np.abs(ref - xr)) <= TOL_F32
    for k in (1, 2, 3, 4, 7, 10, 0):
        got = pkg.sci_twist_tv(to_dev(y), bits, B, tv, 0.05, T, S, fuse_k=k)[0].cpu().numpy()
        np.testing.assert_array_equal(got, ref, err_msg=f"fuse_k={k}")


def test_twist_residual_history(pkg):
    B, nx, ny, T, S = 8, 48, 64, 6, 5
    case, y = make_problem(nx, ny, B, 5, sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    _, _, res = pkg.sci_twist_tv(to_dev(y), bits, B, "atv", 0.05, T, S, resid_every=2)
    want = [O.residual_sq(O.twist_tv(y, case.masks, 0.05, t, S, "atv")[0], y, case.masks) for t in (2, 4, 6)]
    np.testing.assert_allclose(res.cpu().numpy(), want, rtol=1e-4)


def test_twist_first_iteration_is_a_plain_step(pkg):
    """T = 1 returns TVdenoise(Phi^T y + (1/L) Phi^T (y - Phi Phi^T y)): the
    two-step recursion starts after one plain step."""
    B, nx, ny = 4, 40, 30
    case, y = make_problem(nx, ny, B, 9)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    x, _, _ = pkg.sci_twist_tv(to_dev(y), bits, B, "vtv", 0.05, 1, 5)
    x0 = O.adjoint(y, case.masks)
    z = x0 + O.adjoint(y - O.forward(x0, case.masks), case.masks) / O.lipschitz(case.masks)
    assert maxabs(x, O.fgp_prox(z, 0.05, 5, "vtv")) <= TOL_F32


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_twist_16bit_storage(pkg, storage):
    B, nx, ny = 8, 128, 128
    case, y = make_problem(nx, ny, B, 41, sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    x32 = pkg.sci_twist_tv(to_dev(y), bits, B, "itv2d", 0.05, 20, 5)[0].cpu().numpy()
    x16 = pkg.sci_twist_tv(to_dev(y), bits, B, "itv2d", 0.05, 20, 5, storage=storage)[0].cpu().numpy()
    assert abs(O.psnr(x16, case.x_gt) - O.psnr(x32, case.x_gt)) <= 0.1


def test_twist_all_masks_zero(pkg):
    """No pixel measured: L = 0, the gradient step is skipped (1/L taken as 0)
    and x stays the TV-denoised Phi^T y = 0."""
    B, nx, ny = 3, 20, 24
    y = np.random.default_rng(3).random((nx, ny)).astype(np.float32)
    masks = np.zeros((B, nx, ny), np.uint8)
    bits = pkg.sci_masks_pack(to_dev(masks))
    x, _, _ = pkg.sci_twist_tv(to_dev(y), bits, B, "atv", 0.05, 3, 2)
    xr, _ = O.twist_tv(y.astype(np.float64), masks, 0.05, 3, 2, "atv")
    assert maxabs(x, xr) <= TOL_F32
