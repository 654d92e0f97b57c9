"""GPU: degenerate and corrupt inputs, made on the host (no kernel is made to
fault, trap or hang).

- check_input = 1 counts NaN / Inf in y (and theta, u when resuming) on the
  device and returns SCI_ERR_NONFINITE before the solve is enqueued; finite
  inputs give the unchecked result bit for bit;
- without the check a NaN in y reaches the outputs and the FP64 residual
  history (documented behaviour);
- all masks zero (R = 0 everywhere: nothing measured) leaves every outer
  loop finite and equal to the oracle (the pseudo-inverse R^+ = 0);
- one frame with an all-ones mask returns y (to FP32 rounding of theta + (y - theta)).
"""
import numpy as np
import pytest

import oracle as O
from gpu_helpers import TOL_F32, lib, make_problem, maxabs, to_dev

pytestmark = pytest.mark.gpu

NONFINITE = 4


@pytest.fixture(scope="module")
def pkg():
    return lib()


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -float("inf")])
@pytest.mark.parametrize("algo", ["gap", "admm", "fista", "twist"])
def test_check_input_reports_nonfinite_y(pkg, algo, bad):
    B, nx, ny = 4, 40, 56
    case, y = make_problem(nx, ny, B, 3, sigma=0.01)
    y = y.copy()
    y[17, 33] = bad
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    fn = {"gap": pkg.sci_gap_tv, "fista": pkg.sci_fista_tv, "twist": pkg.sci_twist_tv}.get(algo)
    with pytest.raises(pkg.SciError) as e:
        if algo == "admm":
            pkg.sci_admm_tv(to_dev(y), bits, B, "atv", 0.05, 0.01, 3, 2, check_input=True)
        else:
            fn(to_dev(y), bits, B, "atv", 0.05, 3, 2, check_input=True)
    assert e.value.status == NONFINITE


def test_check_input_covers_resumed_state(pkg):
    B, nx, ny = 6, 32, 48
    case, y = make_problem(nx, ny, B, 4, sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    yd = to_dev(y)
    _, th, u, _ = pkg.sci_admm_tv(yd, bits, B, "vtv", 0.05, 0.01, 2, 3)
    th_bad = th.clone()
    th_bad[2, 5, 7] = float("nan")
    with pytest.raises(pkg.SciError) as e:
        pkg.sci_admm_tv(yd, bits, B, "vtv", 0.05, 0.01, 2, 3, theta=th_bad, u=u.clone(), init=False,
                        check_input=True)
    assert e.value.status == NONFINITE
    u_bad = u.clone()
    u_bad[0, 0, 0] = float("inf")
    with pytest.raises(pkg.SciError):
        pkg.sci_admm_tv(yd, bits, B, "vtv", 0.05, 0.01, 2, 3, theta=th.clone(), u=u_bad, init=False,
                        check_input=True)


@pytest.mark.parametrize("tv", ["atv", "vtv"])
def test_check_input_on_finite_data_changes_nothing(pkg, tv):
    B, nx, ny = 8, 64, 72
    case, y = make_problem(nx, ny, B, 6, sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    a = pkg.sci_gap_tv(to_dev(y), bits, B, tv, 0.05, 4, 5)[0].cpu().numpy()
    b = pkg.sci_gap_tv(to_dev(y), bits, B, tv, 0.05, 4, 5, check_input=True)[0].cpu().numpy()
    np.testing.assert_array_equal(a, b)


def test_unchecked_nan_reaches_outputs_and_residuals(pkg):
    B, nx, ny = 4, 32, 32
    case, y = make_problem(nx, ny, B, 8)
    y = y.copy()
    y[3, 4] = float("nan")
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    x, _, res = pkg.sci_gap_tv(to_dev(y), bits, B, "atv", 0.05, 4, 3, resid_every=2)
    assert np.isnan(x.cpu().numpy()).any()
    assert np.isnan(res.cpu().numpy()).all()


@pytest.mark.parametrize("algo", ["gap", "admm", "fista", "twist"])
def test_all_masks_zero(pkg, algo):
    B, nx, ny = 3, 24, 40
    y = np.random.default_rng(5).random((nx, ny)).astype(np.float32)
    masks = np.zeros((B, nx, ny), np.uint8)
    bits = pkg.sci_masks_pack(to_dev(masks))
    yd, y64 = to_dev(y), y.astype(np.float64)
    if algo == "gap":
        x = pkg.sci_gap_tv(yd, bits, B, "itv2d", 0.05, 3, 2)[0]
        xr = O.gap_tv(y64, masks, 0.05, 3, 2, "itv2d")[0]
    elif algo == "admm":
        x = pkg.sci_admm_tv(yd, bits, B, "itv2d", 0.05, 0.01, 3, 2)[0]
        xr = O.admm_tv(y64, masks, 0.05, 0.01, 3, 2, "itv2d")[0]
    elif algo == "fista":
        x = pkg.sci_fista_tv(yd, bits, B, "itv2d", 0.05, 3, 2)[0]
        xr = O.fista_tv(y64, masks, 0.05, 3, 2, "itv2d")[0]
    else:
        x = pkg.sci_twist_tv(yd, bits, B, "itv2d", 0.05, 3, 2)[0]
        xr = O.twist_tv(y64, masks, 0.05, 3, 2, "itv2d")[0]
    assert np.isfinite(x.cpu().numpy()).all()
    assert maxabs(x, xr) <= TOL_F32


@pytest.mark.parametrize("tv", ["atv", "itv2d", "vtv"])
def test_single_frame_all_ones_mask_returns_y(pkg, tv):
    nx, ny = 45, 61
    y = np.random.default_rng(2).random((nx, ny)).astype(np.float32)
    bits = pkg.sci_masks_pack(to_dev(np.ones((1, nx, ny), np.uint8)))
    x = pkg.sci_gap_tv(to_dev(y), bits, 1, tv, 0.05, 5, 4)[0].cpu().numpy()
    np.testing.assert_allclose(x[0], y, rtol=0, atol=1e-6)
