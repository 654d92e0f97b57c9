"""Pins for the oracle's FISTA-TV (Sec. 2.2, FISTA steps).

Readings: L(f) = ||Phi||^2 = max_ij R_ij; standard FISTA momentum with
tau_1 = 1; TVdenoise with the same lam as GAP, so a fixed point minimises
1/2||y - Phi x||^2 + lam L TV(x).  Pins:
- L equals the squared spectral norm of the dense Phi;
- with lam -> 0 the iteration solves the least-squares problem (Phi x = y);
- the converged objective equals an independent SciPy SLSQP solve of that
  problem (ATV, epigraph form).  The minimiser itself need not be unique,
  since Phi has fewer rows than unknowns;
- the first iteration is one projected-gradient step.
"""
import numpy as np
import pytest
from scipy import optimize

import oracle as O


def _dense_phi(C):
    B, nx, ny = C.shape
    n = B * nx * ny
    phi = np.zeros((nx * ny, n))
    for k in range(B):
        for i in range(nx):
            for j in range(ny):
                phi[i * ny + j, (k * nx + i) * ny + j] = C[k, i, j]
    return phi


def _dense_d(B, nx, ny):
    n = B * nx * ny
    rows = []
    for k in range(B):
        for i in range(nx):
            for j in range(ny - 1):
                r = np.zeros(n)
                r[(k * nx + i) * ny + j + 1], r[(k * nx + i) * ny + j] = 1.0, -1.0
                rows.append(r)
    for k in range(B):
        for i in range(nx - 1):
            for j in range(ny):
                r = np.zeros(n)
                r[(k * nx + i + 1) * ny + j], r[(k * nx + i) * ny + j] = 1.0, -1.0
                rows.append(r)
    return np.array(rows)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_lipschitz_is_squared_spectral_norm(seed):
    rng = np.random.default_rng(seed)
    C = (rng.random((4, 5, 6)) < 0.5).astype(np.float64)
    C[:, 0, 0] = 1.0  # at least one pixel with every frame on
    assert O.lipschitz(C) == pytest.approx(np.linalg.norm(_dense_phi(C), 2) ** 2, rel=1e-12)


def test_small_lambda_solves_least_squares():
    rng = np.random.default_rng(4)
    C = (rng.random((3, 5, 6)) < 0.5).astype(np.float64)
    C[0] = np.maximum(C[0], 1.0)  # every pixel measured
    y = O.forward(rng.random((3, 5, 6)), C)
    x, _ = O.fista_tv(y, C, 1e-9, 300, 2, "atv")
    assert np.max(np.abs(O.forward(x, C) - y)) < 1e-6


def scipy_atv_ls_min(C, y, mu):
    """min_x 1/2||y - Phi x||^2 + mu ATV(x) by SciPy SLSQP in epigraph form
    (x and t with -t <= D x <= t, minimise 1/2||.||^2 + mu sum t)."""
    B, nx, ny = C.shape
    phi, d = _dense_phi(C), _dense_d(B, nx, ny)
    n, m = phi.shape[1], d.shape[0]
    yv = y.reshape(-1)

    def f(v):
        r = phi @ v[:n] - yv
        return 0.5 * r @ r + mu * v[n:].sum(), np.concatenate([phi.T @ r, mu * np.ones(m)])

    cons = [{"type": "ineq", "fun": lambda v: v[n:] - d @ v[:n], "jac": lambda v: np.hstack([-d, np.eye(m)])},
            {"type": "ineq", "fun": lambda v: v[n:] + d @ v[:n], "jac": lambda v: np.hstack([d, np.eye(m)])}]
    x0 = O.adjoint(y, C).reshape(-1)
    res = optimize.minimize(f, np.concatenate([x0, np.abs(d @ x0)]), jac=True, constraints=cons,
                            method="SLSQP", options={"ftol": 1e-14, "maxiter": 2000})
    assert res.success
    return res.x[:n].reshape(B, nx, ny)


def atv_ls_objective(x, C, y, mu):
    return 0.5 * float(np.sum((O.forward(x, C) - y) ** 2)) + mu * O.tv_value(x, "atv")


def test_converged_objective_matches_scipy_solve():
    rng = np.random.default_rng(5)
    B, nx, ny = 2, 3, 4
    C = (rng.random((B, nx, ny)) < 0.6).astype(np.float64)
    y = O.forward(rng.random((B, nx, ny)), C)
    lam = 0.05
    mu = lam * O.lipschitz(C)
    ref = atv_ls_objective(scipy_atv_ls_min(C, y, mu), C, y, mu)
    xf, _ = O.fista_tv(y, C, lam, 600, 100, "atv")
    assert abs(atv_ls_objective(xf, C, y, mu) - ref) <= 1e-5 * ref


@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_first_iteration_is_a_gradient_step_then_the_prox(tv):
    rng = np.random.default_rng(6)
    C = (rng.random((3, 6, 5)) < 0.5).astype(np.float64)
    y = O.forward(rng.random((3, 6, 5)), C)
    phi = _dense_phi(C)
    th0 = (phi.T @ y.reshape(-1)).reshape(3, 6, 5)
    z = th0 + (phi.T @ (y.reshape(-1) - phi @ th0.reshape(-1))).reshape(3, 6, 5) / O.lipschitz(C)
    x, _ = O.fista_tv(y, C, 0.05, 1, 5, tv)
    np.testing.assert_allclose(x, O.fgp_prox(z, 0.05, 5, tv), rtol=0, atol=1e-12)
