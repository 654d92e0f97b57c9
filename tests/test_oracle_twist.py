"""Pins for the oracle's TwIST-TV (Sec. 2.2, TwIST steps).

Readings: the unit step runs on the normalised operator Phi / sqrt(L)
(L = max R); alpha and beta follow TwIST's rule from the extreme nonzero
eigenvalues of the normalised Phi^T Phi (xim = 1, xi1 = min_{R>0} R / L);
the first iteration is a plain step; TVdenoise takes lam as for FISTA.  Pins:
- the rule gives the two-step recursion its optimal worst-case rate over
  [xi1, xim]: the largest root modulus of its characteristic polynomial is
  rho there (numpy.roots), and perturbing alpha or beta makes it worse;
- xi1 = xim gives alpha = beta = 1, i.e. plain IST (a dense loop here);
- xi1 is the smallest nonzero eigenvalue of the dense normalised Phi^T Phi;
- lam -> 0 solves the least-squares problem (Phi x = y);
- the converged objective equals an independent SciPy SLSQP solve of
  1/2||y - Phi x||^2 + lam L ATV(x), the problem FISTA-TV also solves;
- a constant ground truth is a fixed point;
- the first two iterations, written out with the dense Phi, catch a swap of
  the x^(t-1) and x^(t) coefficients, which the convergence pins cannot see;
- with xi1 = 1e-4 and no safeguard the plain recursion does not converge on
  the same problem (why the eigenvalue reading is taken).
"""
import numpy as np
import pytest

import oracle as O
from test_oracle_fista import _dense_phi, atv_ls_objective, scipy_atv_ls_min


def _radius(alpha, beta, mu):
    # e^(t+1) = (1 - alpha) e^(t-1) + (alpha - beta mu) e^(t) on an eigenvector
    # of A^T A with eigenvalue mu: roots of r^2 - (alpha - beta mu) r + (alpha - 1)
    return float(np.max(np.abs(np.roots([1.0, -(alpha - beta * mu), alpha - 1.0]))))


@pytest.mark.parametrize("xi1", [1e-4, 0.01, 0.125, 0.5])
def test_params_give_the_optimal_two_step_rate(xi1):
    a, b = O.twist_params(xi1, 1.0)
    r = np.sqrt(xi1)
    rho = (1 - r) / (1 + r)
    grid = np.linspace(xi1, 1.0, 2001)
    worst = max(_radius(a, b, m) for m in grid)
    assert worst == pytest.approx(rho, abs=1e-6)
    assert _radius(a, b, 1.0 + 0.5 * (1 - xi1)) > rho + 1e-3  # outside the interval it is slower
    for da, db in ((0.02, 0.0), (-0.02, 0.0), (0.0, 0.03), (0.0, -0.03)):
        assert max(_radius(a + da, b + db, m) for m in grid) > rho + 1e-4


def test_equal_bounds_give_plain_ist():
    assert O.twist_params(1.0, 1.0) == (1.0, 1.0)
    rng = np.random.default_rng(7)
    C = (rng.random((3, 5, 4)) < 0.5).astype(np.float64)
    y = O.forward(rng.random((3, 5, 4)), C)
    phi, L = _dense_phi(C), O.lipschitz(C)
    x = (phi.T @ y.reshape(-1)).reshape(3, 5, 4)
    for _ in range(6):
        z = x + (phi.T @ (y.reshape(-1) - phi @ x.reshape(-1))).reshape(x.shape) / L
        x = O.fgp_prox(z, 0.05, 4, "itv2d")
    xt, _ = O.twist_tv(y, C, 0.05, 6, 4, "itv2d", xi1=1.0)
    np.testing.assert_allclose(xt, x, atol=1e-12)


@pytest.mark.parametrize("seed", [1, 2])
def test_xi1_is_the_smallest_nonzero_eigenvalue(seed):
    rng = np.random.default_rng(seed)
    C = (rng.random((3, 4, 5)) < 0.5).astype(np.float64)
    C[:, 0, 0] = 1.0
    phi = _dense_phi(C) / np.sqrt(O.lipschitz(C))
    ev = np.linalg.eigvalsh(phi.T @ phi)
    assert ev.max() == pytest.approx(1.0, abs=1e-12)
    assert O.twist_xi1(C) == pytest.approx(ev[ev > 1e-9].min(), abs=1e-12)


def test_small_lambda_solves_least_squares():
    rng = np.random.default_rng(4)
    C = (rng.random((3, 5, 6)) < 0.5).astype(np.float64)
    C[0] = np.maximum(C[0], 1.0)  # every pixel measured
    y = O.forward(rng.random((3, 5, 6)), C)
    x, _ = O.twist_tv(y, C, 1e-9, 100, 2, "atv")
    assert np.max(np.abs(O.forward(x, C) - y)) < 1e-6


def test_converged_objective_matches_scipy_solve():
    rng = np.random.default_rng(5)
    B, nx, ny = 2, 3, 4
    C = (rng.random((B, nx, ny)) < 0.6).astype(np.float64)
    y = O.forward(rng.random((B, nx, ny)), C)
    lam = 0.05
    mu = lam * O.lipschitz(C)
    ref = atv_ls_objective(scipy_atv_ls_min(C, y, mu), C, y, mu)
    xt, _ = O.twist_tv(y, C, lam, 300, 100, "atv")
    assert abs(atv_ls_objective(xt, C, y, mu) - ref) <= 1e-5 * ref
    # the unsafeguarded recursion with xi1 = 1e-4 does not get there
    xb, _ = O.twist_tv(y, C, lam, 300, 100, "atv", xi1=1e-4)
    assert atv_ls_objective(xb, C, y, mu) > 10 * ref


@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_constant_ground_truth_is_a_fixed_point(tv):
    rng = np.random.default_rng(8)
    C = (rng.random((4, 6, 5)) < 0.5).astype(np.float64)
    x_gt = np.full((4, 6, 5), 0.37)
    y = O.forward(x_gt, C)
    x, th = O.twist_tv(y, C, 0.05, 5, 6, tv, theta0=x_gt)
    np.testing.assert_allclose(x, x_gt, atol=1e-13)
    np.testing.assert_allclose(th, x_gt, atol=1e-13)


@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_first_two_iterations_written_out(tv):
    rng = np.random.default_rng(9)
    B, nx, ny = 3, 6, 5
    C = (rng.random((B, nx, ny)) < 0.5).astype(np.float64)
    y = O.forward(rng.random((B, nx, ny)), C)
    phi, L = _dense_phi(C), O.lipschitz(C)
    a, b = O.twist_params(O.twist_xi1(C), 1.0)

    def step(x):
        return x + (phi.T @ (y.reshape(-1) - phi @ x.reshape(-1))).reshape(B, nx, ny) / L

    x0 = (phi.T @ y.reshape(-1)).reshape(B, nx, ny)
    x1 = O.fgp_prox(step(x0), 0.05, 5, tv)
    th1 = O.fgp_prox(step(x1), 0.05, 5, tv)
    x2 = (1 - a) * x0 + (a - b) * x1 + b * th1
    got1, _ = O.twist_tv(y, C, 0.05, 1, 5, tv)
    got2, gth = O.twist_tv(y, C, 0.05, 2, 5, tv)
    np.testing.assert_allclose(got1, x1, atol=1e-12)
    np.testing.assert_allclose(got2, x2, atol=1e-12)
    np.testing.assert_allclose(gth, th1, atol=1e-12)
    assert a != 1.0 and abs((a - b) - (1 - a)) > 0.1  # the two coefficients differ


def test_zero_iterations_return_the_start():
    rng = np.random.default_rng(10)
    C = (rng.random((2, 4, 4)) < 0.5).astype(np.float64)
    y = O.forward(rng.random((2, 4, 4)), C)
    x, th = O.twist_tv(y, C, 0.05, 0, 5, "atv")
    np.testing.assert_array_equal(x, O.adjoint(y, C))
    np.testing.assert_array_equal(th, x)
