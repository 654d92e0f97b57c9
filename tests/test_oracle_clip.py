"""Pins for the oracle's ATV-Clip box (Algorithm 1, ATV-Clip; Sec. 2.3).

Readings: threshold T = lam, step 1/alpha with alpha = 4, output from the
duals after the S-th update.  Pins that do not run the oracle's arithmetic:
- iterates worked out by hand on a one-row, two-pixel image;
- on frames constant along one axis, the converged box is that axis's 1-D
  TV prox: the single-edge closed form (levels move by lam/n1, lam/n2, or
  meet at the mean) and an independent SciPy solve of the ATV dual problem;
- on general inputs, the converged box is x minus the sum of the two 1-D
  corrections: each row's and each column's 1-D prox solved separately by
  SciPy (theta = theta_rows + theta_cols - x);
- invariants: constant frames fixed, per-frame mean kept, |w| <= T,
  transposition swaps the roles of D_h and D_v, flips commute.
A slip that mixes the directions (theta_h used for D_v, or the joint
theta of the FGP box) fails the separable SciPy pin; a threshold of 2 lam or
a missing 1/alpha fails the closed form and the hand iterates.
"""
import numpy as np
import pytest

import oracle as O
from test_oracle_prox import _dual_solve_scipy


def test_hand_iterates_one_row_two_pixels():
    """x = [a, b]: D_h x = b - a, D_h^T w = [-w, w], so theta = [a + w, b - w]
    and w <- clip(w + (theta_1 - theta_0)/4, T)."""
    a, b = 0.2, 0.9
    x = np.array([a, b]).reshape(1, 1, 2)
    # lam = 0.1: w = clip(0.7 / 4 = 0.175, 0.1) = 0.1 at once: theta = [0.3, 0.8]
    np.testing.assert_allclose(O.clip_prox(x, 0.1, 1).reshape(-1), [0.3, 0.8], atol=1e-15)
    np.testing.assert_allclose(O.clip_prox(x, 0.1, 5).reshape(-1), [0.3, 0.8], atol=1e-15)
    # lam = 0.5: w1 = 0.175 -> [0.375, 0.725]; w2 = 0.175 + 0.35/4 = 0.2625 -> [0.4625, 0.6375];
    # w3 = 0.2625 + 0.175/4 = 0.30625 -> [0.50625, 0.59375]
    for S, want in ((1, [0.375, 0.725]), (2, [0.4625, 0.6375]), (3, [0.50625, 0.59375])):
        np.testing.assert_allclose(O.clip_prox(x, 0.5, S).reshape(-1), want, atol=1e-14, err_msg=f"S={S}")
    # converged: |b - a| = 0.7 <= 2 lam, the two pixels meet at the mean
    np.testing.assert_allclose(O.clip_prox(x, 0.5, 200).reshape(-1), [0.55, 0.55], atol=1e-12)


def _step_image(nx, n1, n2, a, b):
    img = np.empty((nx, n1 + n2))
    img[:, :n1] = a
    img[:, n1:] = b
    return img


@pytest.mark.parametrize("a,b,n1,n2,lam", [(0.2, 0.9, 3, 5, 0.3), (0.0, 1.0, 4, 4, 0.5),
                                           (0.4, 0.5, 2, 3, 0.2)])
def test_single_edge_closed_form(a, b, n1, n2, lam):
    nx, B = 4, 2
    x = np.stack([_step_image(nx, n1, n2, a, b)] * B)
    if abs(b - a) > lam * (1.0 / n1 + 1.0 / n2):
        s = np.sign(b - a)
        a2, b2 = a + s * lam / n1, b - s * lam / n2
    else:
        a2 = b2 = (n1 * a + n2 * b) / (n1 + n2)
    want = np.stack([_step_image(nx, n1, n2, a2, b2)] * B)
    np.testing.assert_allclose(O.clip_prox(x, lam, 8000), want, atol=1e-8)
    # the same edge turned by 90 degrees runs through D_v
    np.testing.assert_allclose(O.clip_prox(x.transpose(0, 2, 1), lam, 8000), want.transpose(0, 2, 1),
                               atol=1e-8)


@pytest.mark.parametrize("lam", [0.05, 0.2])
def test_one_axis_inputs_equal_scipy_atv_prox(lam):
    """A frame constant along i: the 2-D ATV prox (SciPy dual solve) is the
    row-wise 1-D prox, which the converged Clip box reproduces."""
    rng = np.random.default_rng(int(lam * 100))
    row = rng.random((2, 1, 6))
    x = np.repeat(row, 4, axis=1)
    np.testing.assert_allclose(O.clip_prox(x, lam, 6000), _dual_solve_scipy(x, lam, "atv"), atol=2e-6)


@pytest.mark.parametrize("lam", [0.05, 0.2])
def test_general_input_is_the_sum_of_separate_1d_proxes(lam):
    rng = np.random.default_rng(7 + int(lam * 100))
    B, nx, ny = 2, 4, 5
    x = rng.random((B, nx, ny))
    rows = np.empty_like(x)
    cols = np.empty_like(x)
    for k in range(B):
        for i in range(nx):
            rows[k, i] = _dual_solve_scipy(x[k:k + 1, i:i + 1, :], lam, "atv").reshape(-1)
        for j in range(ny):
            cols[k, :, j] = _dual_solve_scipy(x[k:k + 1, :, j:j + 1], lam, "atv").reshape(-1)
    np.testing.assert_allclose(O.clip_prox(x, lam, 6000), rows + cols - x, atol=3e-6)
    # which differs from the exact 2-D ATV prox
    assert np.max(np.abs(rows + cols - x - _dual_solve_scipy(x, lam, "atv"))) > 1e-3


@pytest.mark.parametrize("S", [1, 3, 10])
def test_invariants(S):
    lam = 0.07
    x = np.random.default_rng(S).random((3, 7, 6))
    th, (wh, wv) = O.clip_prox(x, lam, S, return_dual=True)
    np.testing.assert_allclose(th.sum(axis=(1, 2)), x.sum(axis=(1, 2)), atol=1e-12)
    assert np.all(np.abs(wh) <= lam) and np.all(np.abs(wv) <= lam)
    assert np.all(wh[:, :, -1] == 0) and np.all(wv[:, -1, :] == 0)
    np.testing.assert_allclose(O.clip_prox(x.transpose(0, 2, 1), lam, S), th.transpose(0, 2, 1), atol=1e-12)
    np.testing.assert_allclose(O.clip_prox(x[:, ::-1, :], lam, S), th[:, ::-1, :], atol=1e-12)
    np.testing.assert_allclose(O.clip_prox(x[:, :, ::-1], lam, S), th[:, :, ::-1], atol=1e-12)
    np.testing.assert_allclose(O.clip_prox(x + 0.3, lam, S), th + 0.3, atol=1e-12)
    const = np.stack([np.full((5, 4), v) for v in (0.1, 0.5, 0.9)])
    np.testing.assert_array_equal(O.clip_prox(const, lam, S), const)


def test_clip_is_atv_only():
    with pytest.raises(ValueError):
        O.clip_prox(np.zeros((1, 2, 2)), 0.1, 2, "itv2d")


@pytest.mark.parametrize("algo", ["gap", "admm"])
def test_outer_loops_take_the_clip_box(algo):
    """dual='clip' in the outer loops runs this box; a noise-free constant
    ground truth stays a fixed point."""
    B, nx, ny = 4, 9, 7
    rng = np.random.default_rng(2)
    C = (rng.random((B, nx, ny)) < 0.5).astype(np.float64)
    x_gt = np.stack([np.full((nx, ny), v) for v in (0.2, 0.4, 0.6, 0.8)])
    y = O.forward(x_gt, C)
    if algo == "gap":
        x, th = O.gap_tv(y, C, 0.05, 4, 3, "atv", theta0=x_gt, dual="clip")
    else:
        x, th, _ = O.admm_tv(y, C, 0.05, 0.01, 4, 3, "atv", theta0=x_gt, dual="clip")
    np.testing.assert_allclose(th, x_gt, atol=1e-13)
    np.testing.assert_allclose(x, x_gt, atol=1e-13)
    y2 = O.forward(rng.random((B, nx, ny)), C)
    x1, th1 = O.gap_tv(y2, C, 0.05, 1, 3, "atv", dual="clip")
    np.testing.assert_allclose(th1, O.clip_prox(O.gap_project(O.adjoint(y2, C), y2, C), 0.05, 3), atol=1e-14)
