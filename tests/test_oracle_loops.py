"""Pins for the oracle's GAP-TV and ADMM-TV outer loops (Eqs. 21-26; Algorithm 1)."""
import numpy as np
import pytest

import oracle as O
import sci_synth as ss


@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_constant_ground_truth_is_fixed_point(tv):
    """Noise-free y from a constant video: theta = x_gt gives Phi theta = y, so
    the projection returns theta and the prox of a constant frame is itself."""
    B, nx, ny = 4, 9, 7
    C = ss.masks_bernoulli(nx, ny, B, 3).astype(np.float64)
    x_gt = np.stack([np.full((nx, ny), v) for v in (0.2, 0.4, 0.6, 0.8)])
    y = O.forward(x_gt, C)
    x, th = O.gap_tv(y, C, 0.05, 5, 3, tv, theta0=x_gt)
    np.testing.assert_allclose(th, x_gt, atol=1e-14)
    np.testing.assert_allclose(x, x_gt, atol=1e-14)
    x, th, u = O.admm_tv(y, C, 0.05, 0.01, 5, 3, tv, theta0=x_gt)
    np.testing.assert_allclose(th, x_gt, atol=1e-13)
    np.testing.assert_allclose(u, 0.0, atol=1e-13)


@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_single_frame_all_ones_mask_returns_y(tv):
    """B = 1 with C = 1: Phi = I, the projection returns y exactly."""
    rng = np.random.default_rng(4)
    y = rng.random((6, 5))
    C = np.ones((1, 6, 5))
    for T in (1, 3, 7):
        x, _ = O.gap_tv(y, C, 0.1, T, 4, tv)
        np.testing.assert_allclose(x[0], y, atol=1e-15)


@pytest.mark.parametrize("algo", ["gap", "admm"])
@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_resume_equals_single_run(algo, tv):
    case = ss.make_case(12, 10, 3, 5, sigma=0.01)
    C = case.masks.astype(np.float64)
    y = O.forward(case.x_gt, C) + case.noise
    if algo == "gap":
        x_full, th_full = O.gap_tv(y, C, 0.05, 7, 3, tv)
        _, th1 = O.gap_tv(y, C, 0.05, 4, 3, tv)
        x2, th2 = O.gap_tv(y, C, 0.05, 3, 3, tv, theta0=th1)
    else:
        x_full, th_full, _ = O.admm_tv(y, C, 0.05, 0.01, 7, 3, tv)
        _, th1, u1 = O.admm_tv(y, C, 0.05, 0.01, 4, 3, tv)
        x2, th2, _ = O.admm_tv(y, C, 0.05, 0.01, 3, 3, tv, theta0=th1, u0=u1)
    np.testing.assert_array_equal(x2, x_full)
    np.testing.assert_array_equal(th2, th_full)


@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_gap_output_is_feasible(tv):
    """x^(T) is a projection output: Phi x = y on every pixel with R > 0."""
    case = ss.make_case(16, 12, 5, 6, sigma=0.01)
    C = case.masks.astype(np.float64)
    y = O.forward(case.x_gt, C) + case.noise
    x, _ = O.gap_tv(y, C, 0.05, 4, 3, tv)
    R = O.mask_energy(C)
    np.testing.assert_allclose(O.forward(x, C)[R > 0], y[R > 0], atol=1e-12)


def test_admm_u_is_running_sum_of_residuals():
    """u^(T) = sum_t (x^(t) - theta^(t)) from u^(0) = 0 (Eq. 26)."""
    case = ss.make_case(10, 10, 4, 7, sigma=0.01)
    C = case.masks.astype(np.float64)
    y = O.forward(case.x_gt, C) + case.noise
    th = O.adjoint(y, C)
    u = np.zeros_like(th)
    acc = np.zeros_like(th)
    for _ in range(4):
        x = O.admm_xupdate(th, u, y, C, 0.01)
        th = O.fgp_prox(u + x, 0.05, 3, "vtv")
        acc += x - th
        u = u + x - th
    _, th_o, u_o = O.admm_tv(y, C, 0.05, 0.01, 4, 3, "vtv")
    np.testing.assert_allclose(u_o, acc, atol=1e-13)
    np.testing.assert_allclose(th_o, th, atol=1e-13)


@pytest.mark.parametrize("algo", ["gap", "admm"])
def test_psnr_rises_then_plateaus(algo):
    """Qualitative trend of Sec. 3 (PSNR grows with iterations, GAP best near 60)."""
    case = ss.make_case(64, 64, 8, 1)
    C = case.masks.astype(np.float64)
    y = O.forward(case.x_gt, C)
    ps = []
    for T in (1, 10, 40):
        if algo == "gap":
            x, _ = O.gap_tv(y, C, 0.05, T, 5, "atv")
        else:
            x, _, _ = O.admm_tv(y, C, 0.05, 0.01, T, 5, "atv")
        ps.append(O.psnr(x, case.x_gt))
    assert ps[0] < ps[1] < ps[2] + 0.5
    assert ps[2] > O.psnr(O.adjoint(y, C), case.x_gt) + 3.0
