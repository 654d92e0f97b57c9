"""Pins for the oracle's measurement model, projection and ADMM x-update.

Each check compares the oracle with something other than itself: the dense
sensing matrix built from Eq. 2, numpy's SVD pseudo-inverse and dense linear
solves, and hand-computed values.
"""
import itertools

import numpy as np
import pytest

import oracle as O


def dense_phi(C):
    """Phi = [D_1, ..., D_B] with D_k = diag(vec C_k) (Eq. 2), row-major vec."""
    B, nx, ny = C.shape
    n = nx * ny
    Phi = np.zeros((n, n * B))
    for k in range(B):
        Phi[:, k * n:(k + 1) * n] = np.diag(C[k].reshape(-1))
    return Phi


SHAPES = [(2, 3, 1), (3, 2, 2), (4, 5, 3), (5, 5, 4)]


@pytest.mark.parametrize("nx,ny,B", SHAPES)
def test_forward_adjoint_match_dense_phi(nx, ny, B):
    rng = np.random.default_rng(10 + nx * 7 + B)
    C = rng.normal(size=(B, nx, ny))
    x = rng.normal(size=(B, nx, ny))
    y = rng.normal(size=(nx, ny))
    Phi = dense_phi(C)
    np.testing.assert_allclose(O.forward(x, C).reshape(-1), Phi @ x.reshape(-1), rtol=0, atol=1e-12)
    np.testing.assert_allclose(O.adjoint(y, C).reshape(-1), Phi.T @ y.reshape(-1), rtol=0, atol=1e-12)
    # dot-product test <Phi x, y> = <x, Phi^T y>
    lhs = float(np.sum(O.forward(x, C) * y))
    rhs = float(np.sum(x * O.adjoint(y, C)))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


@pytest.mark.parametrize("nx,ny,B", SHAPES)
def test_phi_phit_is_diag_R(nx, ny, B):
    rng = np.random.default_rng(3 + B)
    C = rng.normal(size=(B, nx, ny))
    Phi = dense_phi(C)
    np.testing.assert_allclose(Phi @ Phi.T, np.diag(O.mask_energy(C).reshape(-1)), atol=1e-12)


def _binary_case(nx, ny, B, seed, zero_pixels=2):
    rng = np.random.default_rng(seed)
    C = (rng.random((B, nx, ny)) < 0.5).astype(np.float64)
    # force some all-zero pixels (R = 0) and one all-one pixel
    flat = C.reshape(B, -1)
    flat[:, :zero_pixels] = 0.0
    flat[:, -1] = 1.0
    theta = rng.normal(size=(B, nx, ny))
    y = rng.normal(size=(nx, ny))
    return C, theta, y


@pytest.mark.parametrize("nx,ny,B", [(3, 3, 2), (4, 5, 3), (5, 4, 4)])
def test_gap_projection_equals_pinv(nx, ny, B):
    C, theta, y = _binary_case(nx, ny, B, 100 + nx)
    Phi = dense_phi(C)
    want = theta.reshape(-1) + np.linalg.pinv(Phi) @ (y.reshape(-1) - Phi @ theta.reshape(-1))
    x = O.gap_project(theta, y, C)
    np.testing.assert_allclose(x.reshape(-1), want, atol=1e-10)


@pytest.mark.parametrize("nx,ny,B", [(3, 3, 2), (4, 5, 3), (6, 6, 8)])
def test_gap_projection_properties(nx, ny, B):
    C, theta, y = _binary_case(nx, ny, B, 7 * nx + B)
    R = O.mask_energy(C)
    x = O.gap_project(theta, y, C)
    # feasibility on R > 0 pixels, unchanged voxels on R = 0 pixels
    np.testing.assert_allclose(O.forward(x, C)[R > 0], y[R > 0], atol=1e-12)
    np.testing.assert_array_equal(x[:, R == 0], theta[:, R == 0])
    # idempotent
    np.testing.assert_allclose(O.gap_project(x, y, C), x, atol=1e-12)
    # closest point: any other feasible point is farther from theta
    rng = np.random.default_rng(5)
    for _ in range(5):
        z = O.gap_project(x + rng.normal(size=x.shape), y, C)
        z[:, R == 0] = x[:, R == 0] + rng.normal(size=z[:, R == 0].shape)
        assert np.linalg.norm(z - theta) >= np.linalg.norm(x - theta) - 1e-12


@pytest.mark.parametrize("rho", [0.01, 0.5, 3.0])
def test_admm_xupdate_equals_dense_solve(rho):
    C, theta, y = _binary_case(4, 3, 3, 77)
    rng = np.random.default_rng(78)
    u = rng.normal(size=theta.shape)
    Phi = dense_phi(C)
    A = Phi.T @ Phi + rho * np.eye(Phi.shape[1])
    b = Phi.T @ y.reshape(-1) + rho * (theta - u).reshape(-1)
    want = np.linalg.solve(A, b)
    np.testing.assert_allclose(O.admm_xupdate(theta, u, y, C, rho).reshape(-1), want, atol=1e-10)


def test_admm_xupdate_rho0_is_gap_projection_of_v():
    """At rho = 0 the ADMM x-update degrades to the GAP projection (Sec. 2.2)."""
    C, theta, y = _binary_case(5, 4, 4, 21)
    u = np.random.default_rng(22).normal(size=theta.shape)
    Phi = dense_phi(C)
    v = (theta - u).reshape(-1)
    want = v + np.linalg.pinv(Phi) @ (y.reshape(-1) - Phi @ v)
    np.testing.assert_allclose(O.admm_xupdate(theta, u, y, C, 0.0).reshape(-1), want, atol=1e-10)


def test_forward_hand_values():
    # y_ij = sum_k c_ijk x_ijk (Eq. 4) on a 1x2 image with 2 frames
    x = np.array([[[1.0, 2.0]], [[3.0, 4.0]]])
    C = np.array([[[1.0, 0.0]], [[1.0, 1.0]]])
    np.testing.assert_array_equal(O.forward(x, C), [[4.0, 4.0]])
    np.testing.assert_array_equal(O.mask_energy(C), [[2.0, 1.0]])
    # projection of theta = 0 onto y = [[2, 3]]: r = y / R = [1, 3]
    x = O.gap_project(np.zeros((2, 1, 2)), np.array([[2.0, 3.0]]), C)
    np.testing.assert_array_equal(x, [[[1.0, 0.0]], [[1.0, 3.0]]])


@pytest.mark.parametrize("nx,ny", [(1, 1), (1, 4), (4, 1), (3, 5), (6, 2)])
def test_gradients_match_dense_eq7(nx, ny):
    """D_h in R^{(ny-1) x ny}, D_v in R^{(nx-1) x nx}: D_h x_k = X_k D_h^T, D_v x_k = D_v X_k."""
    def diffmat(n):
        D = np.zeros((max(n - 1, 0), n))
        for r in range(n - 1):
            D[r, r], D[r, r + 1] = -1.0, 1.0
        return D
    rng = np.random.default_rng(nx * 10 + ny)
    B = 2
    X = rng.normal(size=(B, nx, ny))
    Dh, Dv = diffmat(ny), diffmat(nx)
    gh, gv = O.grad_h(X), O.grad_v(X)
    for k in range(B):
        np.testing.assert_allclose(gh[k][:, :ny - 1], X[k] @ Dh.T, atol=1e-14)
        np.testing.assert_allclose(gv[k][:nx - 1, :], Dv @ X[k], atol=1e-14)
    assert np.all(gh[:, :, ny - 1] == 0) and np.all(gv[:, nx - 1, :] == 0)
    # adjoints against the dense transposes
    Wh = rng.normal(size=(B, nx, ny))
    Wv = rng.normal(size=(B, nx, ny))
    ah, av = O.grad_h_adj(Wh), O.grad_v_adj(Wv)
    for k in range(B):
        np.testing.assert_allclose(ah[k], Wh[k][:, :ny - 1] @ Dh, atol=1e-14)
        np.testing.assert_allclose(av[k], Dv.T @ Wv[k][:nx - 1, :], atol=1e-14)


def test_tv_hand_values():
    x = np.array([[[0.0, 1.0], [2.0, 4.0]]])
    # gh = [[1,0],[2,0]], gv = [[2,3],[0,0]]
    assert O.tv_value(x, "atv") == pytest.approx(8.0, abs=1e-14)
    assert O.tv_value(x, "itv2d") == pytest.approx(np.sqrt(5.0) + 3.0 + 2.0, abs=1e-14)
    x2 = np.concatenate([x, 2.0 * x], axis=0)
    # per pixel sqrt(sum over both frames): sqrt(5+20), sqrt(9+36), sqrt(4+16)
    assert O.tv_value(x2, "vtv") == pytest.approx(5.0 + np.sqrt(45.0) + np.sqrt(20.0), abs=1e-13)
    assert O.tv_value(x2, "itv2d") == pytest.approx(3.0 * (np.sqrt(5.0) + 5.0), abs=1e-13)


def test_dual_project_hand_values():
    ah = np.array([[[3.0, 0.5]], [[0.0, -2.0]]])
    av = np.array([[[4.0, 0.0]], [[0.0, 0.0]]])
    ph, pv = O.dual_project(ah, av, "atv")
    np.testing.assert_array_equal(ph, [[[1.0, 0.5]], [[0.0, -1.0]]])
    np.testing.assert_array_equal(pv, [[[1.0, 0.0]], [[0.0, 0.0]]])
    ph, pv = O.dual_project(ah, av, "itv2d")
    np.testing.assert_allclose(ph, [[[0.6, 0.5]], [[0.0, -1.0]]], atol=1e-15)
    np.testing.assert_allclose(pv, [[[0.8, 0.0]], [[0.0, 0.0]]], atol=1e-15)
    ph, pv = O.dual_project(ah, av, "vtv")
    # pixel 0: sqrt(9+16+0) = 5 ; pixel 1: sqrt(0.25 + 4) = sqrt(4.25)
    s = np.sqrt(4.25)
    np.testing.assert_allclose(ph, [[[0.6, 0.5 / s]], [[0.0, -2.0 / s]]], atol=1e-15)
    np.testing.assert_allclose(pv, [[[0.8, 0.0]], [[0.0, 0.0]]], atol=1e-15)


def test_momentum_coefficients_hand_values():
    c = O.fgp_momentum_coeffs(3)
    nu1 = (1 + np.sqrt(5.0)) / 2
    nu2 = (1 + np.sqrt(1 + 4 * nu1 ** 2)) / 2
    nu3 = (1 + np.sqrt(1 + 4 * nu2 ** 2)) / 2
    assert c[0] == 0.0
    assert c[1] == pytest.approx((nu1 - 1) / nu2, abs=1e-15)
    assert c[2] == pytest.approx((nu2 - 1) / nu3, abs=1e-15)
    assert c[1] == pytest.approx(0.2817535251, abs=1e-9)


def test_all_index_orders_consistent():
    """Frame-major [B][nx][ny]: masks multiply their own frame only."""
    B, nx, ny = 3, 2, 2
    for k, i, j in itertools.product(range(B), range(nx), range(ny)):
        x = np.zeros((B, nx, ny))
        C = np.zeros((B, nx, ny))
        x[k, i, j] = 2.0
        C[k, i, j] = 3.0
        y = O.forward(x, C)
        assert y[i, j] == 6.0 and np.sum(y) == 6.0
