"""Pins for the oracle's GAP-TV and ADMM-TV outer loops (Eqs. 21-26; Algorithm 1).

Besides fixed points, feasibility and resume, two pins check how each loop
wires its steps together, from references that share no code with the
oracle's loops:
- the first two GAP-TV and ADMM-TV iterations written out with a dense
  pseudo-inverse (GAP, Eq. 21) or a dense solve of the normal equations
  (ADMM, Eq. 24) and the exact TV prox from an independent SciPy solve of its
  dual problem, against the oracle run with enough FGP updates to converge;
- the ADMM fixed point: with TVdenoise at the same lam as GAP (Eq. 25 read
  without rho), a converged run has x = theta and rho u = Phi^T (y - Phi x),
  so x minimises 1/2||y - Phi x||^2 + rho lam TV(x); that minimum is found
  by an independent SciPy solve in epigraph form.
"""
import numpy as np
import pytest
from scipy import optimize

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


# ------------------------------------------------ wiring: first two iterations

from test_oracle_fista import _dense_d, _dense_phi  # noqa: E402
from test_oracle_prox import _dual_solve_scipy  # noqa: E402

S_CONVERGED = 3000  # FGP updates: the oracle's prox then agrees with SciPy's to ~1e-7


def _small_problem(seed):
    rng = np.random.default_rng(seed)
    B, nx, ny = 2, 4, 4
    C = (rng.random((B, nx, ny)) < 0.5).astype(np.float64)
    C[:, 0, 0] = 0.0  # one unmeasured pixel: the pseudo-inverse's R = 0 case
    x_gt = rng.random((B, nx, ny))
    y = O.forward(x_gt, C) + 0.02 * rng.standard_normal((nx, ny))
    return C, y


@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_gap_first_two_iterations_written_out(tv):
    """x^(t) = theta + pinv(Phi)(y - Phi theta) (Eq. 21) with the dense
    pseudo-inverse, theta^(t) = prox_{lam TV}(x^(t)) from the SciPy dual solve;
    denoising theta instead of x (or skipping the projection) fails here."""
    C, y = _small_problem({"atv": 21, "itv2d": 22, "vtv": 23}[tv])
    lam = 0.15
    phi = _dense_phi(C)
    pinv = np.linalg.pinv(phi)
    shape = C.shape
    theta = (phi.T @ y.reshape(-1)).reshape(shape)  # theta^(0) = Phi^T y
    xs, ths = [], []
    for _ in range(2):
        x = theta + (pinv @ (y.reshape(-1) - phi @ theta.reshape(-1))).reshape(shape)
        theta = _dual_solve_scipy(x, lam, tv)
        xs.append(x)
        ths.append(theta)
    for T in (1, 2):
        x_o, th_o = O.gap_tv(y, C, lam, T, S_CONVERGED, tv)
        np.testing.assert_allclose(x_o, xs[T - 1], atol=1e-5, err_msg=f"x^({T})")
        np.testing.assert_allclose(th_o, ths[T - 1], atol=1e-5, err_msg=f"theta^({T})")


@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_admm_first_two_iterations_written_out(tv):
    """x = solve(Phi^T Phi + rho I, Phi^T y + rho (theta - u)) (Eq. 24),
    theta = prox_{lam TV}(u + x) (Eq. 25), u = u + x - theta (Eq. 26), by a
    dense solve and the SciPy dual solve; denoising x instead of u + x fails
    at the second iteration, where u is no longer zero."""
    C, y = _small_problem({"atv": 31, "itv2d": 32, "vtv": 33}[tv])
    lam, rho = 0.15, 0.3
    phi = _dense_phi(C)
    n = phi.shape[1]
    shape = C.shape
    theta = (phi.T @ y.reshape(-1)).reshape(shape)
    u = np.zeros(shape)
    hist = []
    for _ in range(2):
        rhs = phi.T @ y.reshape(-1) + rho * (theta - u).reshape(-1)
        x = np.linalg.solve(phi.T @ phi + rho * np.eye(n), rhs).reshape(shape)
        theta = _dual_solve_scipy(u + x, lam, tv)
        u = u + x - theta
        hist.append((x, theta, u))
    assert np.max(np.abs(hist[0][2])) > 1e-3  # u^(1) != 0, so iteration 2 tells u + x from x
    for T in (1, 2):
        x_o, th_o, u_o = O.admm_tv(y, C, lam, rho, T, S_CONVERGED, tv)
        x_w, th_w, u_w = hist[T - 1]
        np.testing.assert_allclose(x_o, x_w, atol=1e-5, err_msg=f"x^({T})")
        np.testing.assert_allclose(th_o, th_w, atol=1e-5, err_msg=f"theta^({T})")
        np.testing.assert_allclose(u_o, u_w, atol=1e-5, err_msg=f"u^({T})")


# ------------------------------------------------ wiring: the ADMM fixed point

def _pair_index(B, nx, ny):
    """Rows of the dense D (test_oracle_fista._dense_d: all D_h rows, then all
    D_v rows) that belong to each TV group: one row per difference (ATV), the
    h and v differences of a voxel (ITV2D), those of all frames of a pixel (VTV)."""
    nh = B * nx * (ny - 1)
    h_row, v_row = {}, {}
    r = 0
    for k in range(B):
        for i in range(nx):
            for j in range(ny - 1):
                h_row[(k, i, j)] = r
                r += 1
    for k in range(B):
        for i in range(nx - 1):
            for j in range(ny):
                v_row[(k, i, j)] = r
                r += 1
    assert r - nh == B * (nx - 1) * ny
    return h_row, v_row


def _tv_groups(tv, B, nx, ny):
    h_row, v_row = _pair_index(B, nx, ny)
    groups = []
    if tv == "atv":
        return [[r] for r in sorted(list(h_row.values()) + list(v_row.values()))]
    for i in range(nx):
        for j in range(ny):
            if tv == "itv2d":
                for k in range(B):
                    g = [m[(k, i, j)] for m in (h_row, v_row) if (k, i, j) in m]
                    if g:
                        groups.append(g)
            else:
                g = [m[(k, i, j)] for k in range(B) for m in (h_row, v_row) if (k, i, j) in m]
                if g:
                    groups.append(g)
    return groups


def scipy_tv_ls_min(C, y, mu, tv):
    """min_x 1/2||y - Phi x||^2 + mu TV(x) by SciPy SLSQP in epigraph form:
    variables x and one t per TV group, objective 1/2||.||^2 + mu sum t, with
    dense Phi and D from Eqs. 2 and 7 and nothing from the oracle but the
    problem data.  ATV: -t <= D x <= t (linear).  ITV2D / VTV:
    t_g >= sqrt(||(D x)_g||^2 + delta^2) with delta = 1e-9, a smooth cone
    (the exact cone's gradient is undefined at its apex, where many groups
    of a TV minimiser sit); it moves the optimal value by at most
    mu * (number of groups) * delta."""
    B, nx, ny = C.shape
    phi, d = _dense_phi(C), _dense_d(B, nx, ny)
    n = phi.shape[1]
    groups = _tv_groups(tv, B, nx, ny)
    m = len(groups)
    yv = y.reshape(-1)
    delta = 1e-9

    def f(v):
        r = phi @ v[:n] - yv
        return 0.5 * r @ r + mu * v[n:].sum(), np.concatenate([phi.T @ r, mu * np.ones(m)])

    if tv == "atv":
        rows = np.array([g[0] for g in groups])
        dg = d[rows]
        cons = [{"type": "ineq", "fun": lambda v: v[n:] - dg @ v[:n],
                 "jac": lambda v: np.hstack([-dg, np.eye(m)])},
                {"type": "ineq", "fun": lambda v: v[n:] + dg @ v[:n],
                 "jac": lambda v: np.hstack([dg, np.eye(m)])}]
    else:
        def cone(v):
            dx = d @ v[:n]
            return np.array([v[n + g] - np.sqrt(np.sum(dx[rows] ** 2) + delta * delta)
                             for g, rows in enumerate(groups)])

        def cone_jac(v):
            dx = d @ v[:n]
            J = np.zeros((m, n + m))
            for g, rows in enumerate(groups):
                nrm = np.sqrt(np.sum(dx[rows] ** 2) + delta * delta)
                J[g, :n] = -(dx[rows] @ d[rows]) / nrm
                J[g, n + g] = 1.0
            return J
        cons = [{"type": "ineq", "fun": cone, "jac": cone_jac}]

    x0 = O.adjoint(y, C).reshape(-1)
    dx0 = d @ x0
    t0 = np.array([np.sqrt(np.sum(dx0[rows] ** 2)) + 1e-3 for rows in groups])
    res = optimize.minimize(f, np.concatenate([x0, t0]), jac=True, method="SLSQP", constraints=cons,
                            options={"ftol": 1e-12, "maxiter": 5000})
    assert res.success, res.message
    return res.x[:n].reshape(B, nx, ny)


def tv_ls_objective(x, C, y, mu, tv):
    return 0.5 * float(np.sum((O.forward(x, C) - y) ** 2)) + mu * O.tv_value(x, tv)


@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_converged_admm_minimises_rho_lambda_tv_problem(tv):
    """A converged ADMM-TV run (Eqs. 24-26, TVdenoise at lam) has x = theta
    and minimises 1/2||y - Phi x||^2 + rho lam TV(x): its objective equals the
    SciPy minimum.  The minimiser need not be unique (Phi has a nullspace and
    TV is not strictly convex), but Phi x* is (the data term is strictly
    convex in Phi x), and so is TV(x*); both are compared."""
    rng = np.random.default_rng({"atv": 41, "itv2d": 42, "vtv": 43}[tv])
    B, nx, ny = 2, 3, 4
    C = (rng.random((B, nx, ny)) < 0.6).astype(np.float64)
    y = O.forward(rng.random((B, nx, ny)), C)
    # rho = 2 with lam = 0.05 (rho lam = 0.1): the fixed point of 300 FGP
    # updates from w = 0 then lies within ~2e-6 (relative) of the exact one
    lam, rho = 0.05, 2.0
    mu = rho * lam
    x_ref = scipy_tv_ls_min(C, y, mu, tv)
    f_ref = tv_ls_objective(x_ref, C, y, mu, tv)
    x, th, _ = O.admm_tv(y, C, lam, rho, 200, 300, tv)
    np.testing.assert_allclose(x, th, atol=1e-6)  # converged: x = theta
    f_admm = tv_ls_objective(x, C, y, mu, tv)
    assert abs(f_admm - f_ref) <= 5e-6 * f_ref, (f_admm, f_ref)
    np.testing.assert_allclose(O.forward(x, C), O.forward(x_ref, C), atol=1e-4)
    assert O.tv_value(x, tv) == pytest.approx(O.tv_value(x_ref, tv), rel=1e-4, abs=1e-6)
    # the GAP/TVdenoise-strength slip (prox at lam / rho, Eq. 25 read with rho)
    # converges to a different problem's minimiser
    x_alt, _, _ = O.admm_tv(y, C, lam / rho, rho, 200, 300, tv)
    assert tv_ls_objective(x_alt, C, y, mu, tv) > f_ref * (1 + 1e-3)
