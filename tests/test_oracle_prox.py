"""Pins for the oracle's FGP TV proximal map (Algorithm 1, ATV-FGP box; Eqs. 29-32).

Pins: hand-computed FGP iterates on a 1x2 image (tests/golden/fgp_1x2.json),
an independent SciPy solve of the dual problem on 4x4x2 inputs, the closed
form of TV denoising for a single straight edge, the duality gap, and exact
invariants of every finite-S iterate.
"""
import json
import os

import numpy as np
import pytest
from scipy import optimize

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_fgp_hand_iterates_golden():
    with open(os.path.join(GOLDEN, "fgp_1x2.json")) as f:
        g = json.load(f)
    x = np.array(g["x"], dtype=np.float64).reshape(1, 1, 2)
    for case in g["cases"]:
        th = O.fgp_prox(x, case["lam"], case["S"], case["tv"])
        np.testing.assert_allclose(th.reshape(-1), case["theta"], atol=1e-9,
                                   err_msg=str(case))
    v = g["vtv_two_frames"]
    x2 = np.array(v["x"], dtype=np.float64).reshape(2, 1, 2)
    th = O.fgp_prox(x2, v["lam"], v["S"], "vtv")
    np.testing.assert_allclose(th.reshape(2, 2), v["theta"], atol=1e-10)


# ---------------------------------------------------------------- SciPy dual solve

def _dual_solve_scipy(x, lam, tv, return_w=False):
    """min_w 1/2||x - lam D^T w||^2 over the TV's dual unit set, by SciPy.

    Variables are the non-padded dual entries only.  theta* = x - lam D^T w*;
    return_w=True returns (theta*, (w_h*, w_v*)).
    """
    B, nx, ny = x.shape
    mh = np.zeros((B, nx, ny), bool)
    mh[:, :, :ny - 1] = True
    mv = np.zeros((B, nx, ny), bool)
    mv[:, :nx - 1, :] = True
    nh, nv = int(mh.sum()), int(mv.sum())

    def unpack(z):
        wh = np.zeros((B, nx, ny))
        wv = np.zeros((B, nx, ny))
        wh[mh] = z[:nh]
        wv[mv] = z[nh:]
        return wh, wv

    def f(z):
        wh, wv = unpack(z)
        t = x - lam * O.div_adj(wh, wv)
        # gradient: -lam * D t restricted to the variables
        gh = -lam * O.grad_h(t)
        gv = -lam * O.grad_v(t)
        return 0.5 * float(np.sum(t * t)), np.concatenate([gh[mh], gv[mv]])

    z0 = np.zeros(nh + nv)
    if tv == "atv":
        res = optimize.minimize(f, z0, jac=True, method="L-BFGS-B",
                                bounds=[(-1.0, 1.0)] * (nh + nv),
                                options=dict(ftol=1e-16, gtol=1e-13, maxiter=20000, maxcor=50))
    else:
        def cons(z):
            wh, wv = unpack(z)
            if tv == "itv2d":
                return (1.0 - wh * wh - wv * wv).reshape(-1)
            return (1.0 - np.sum(wh * wh + wv * wv, axis=0)).reshape(-1)
        res = optimize.minimize(f, z0, jac=True, method="SLSQP",
                                constraints=[dict(type="ineq", fun=cons)],
                                options=dict(ftol=1e-15, maxiter=2000))
    wh, wv = unpack(res.x)
    theta = x - lam * O.div_adj(wh, wv)
    return (theta, (wh, wv)) if return_w else theta


@pytest.mark.parametrize("tv", O.TV_TYPES)
@pytest.mark.parametrize("lam", [0.05, 0.2])
def test_converged_fgp_matches_scipy_dual_solve(tv, lam):
    rng = np.random.default_rng({"atv": 1, "itv2d": 2, "vtv": 3}[tv] + int(lam * 100))
    x = rng.random((2, 4, 4))
    th_fgp = O.fgp_prox(x, lam, 4000, tv)
    th_ref = _dual_solve_scipy(x, lam, tv)
    np.testing.assert_allclose(th_fgp, th_ref, atol=2e-6)
    # the FGP point is at least as good as SciPy's in the primal objective
    assert O.prox_objective(th_fgp, x, lam, tv) <= O.prox_objective(th_ref, x, lam, tv) + 1e-9


@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_duality_gap_closes(tv):
    rng = np.random.default_rng(11)
    x = rng.random((3, 6, 5))
    lam = 0.1
    gaps = []
    for S in (10, 100, 2000):
        th, (ph, pv) = O.fgp_prox(x, lam, S, tv, return_dual=True)
        gap = O.prox_objective(th, x, lam, tv) - O.dual_objective(ph, pv, x, lam)
        assert gap >= -1e-12
        gaps.append(gap)
    assert gaps[1] < gaps[0] and gaps[2] < 1e-6 * max(1.0, gaps[0])


# ---------------------------------------------------------------- closed form

def _step_image(nx, n1, n2, a, b):
    img = np.empty((nx, n1 + n2))
    img[:, :n1] = a
    img[:, n1:] = b
    return img


@pytest.mark.parametrize("tv", O.TV_TYPES)
@pytest.mark.parametrize("a,b,n1,n2,lam", [(0.2, 0.9, 3, 5, 0.3), (0.0, 1.0, 4, 4, 0.5),
                                           (0.4, 0.5, 2, 3, 0.2)])
def test_prox_of_single_edge_closed_form(tv, a, b, n1, n2, lam):
    """An image constant along rows with one vertical edge keeps its edge; the
    levels move toward each other by lam/n1 and lam/n2 (or merge at the mean).
    With B identical frames VTV scales lam by 1/sqrt(B); ATV/ITV2D act per frame.
    """
    nx, B = 4, 3
    x = np.stack([_step_image(nx, n1, n2, a, b)] * B)
    leff = lam / np.sqrt(B) if tv == "vtv" else lam
    if abs(b - a) > leff * (1.0 / n1 + 1.0 / n2):
        s = np.sign(b - a)
        a2, b2 = a + s * leff / n1, b - s * leff / n2
    else:
        a2 = b2 = (n1 * a + n2 * b) / (n1 + n2)
    want = np.stack([_step_image(nx, n1, n2, a2, b2)] * B)
    got = O.fgp_prox(x, lam, 6000, tv)
    np.testing.assert_allclose(got, want, atol=1e-8)


# ---------------------------------------------------------------- invariants

def _rand(seed, shape=(3, 7, 6)):
    return np.random.default_rng(seed).random(shape)


@pytest.mark.parametrize("tv", O.TV_TYPES)
@pytest.mark.parametrize("S", [1, 2, 5, 10])
def test_fgp_invariants(tv, S):
    lam = 0.05
    x = _rand(S)
    th, (ph, pv) = O.fgp_prox(x, lam, S, tv, return_dual=True)
    # per-frame mean preserved: 1^T D^T = 0
    np.testing.assert_allclose(th.sum(axis=(1, 2)), x.sum(axis=(1, 2)), atol=1e-12)
    # dual feasibility
    if tv == "atv":
        assert np.all(np.abs(ph) <= 1 + 1e-15) and np.all(np.abs(pv) <= 1 + 1e-15)
    elif tv == "itv2d":
        assert np.all(ph * ph + pv * pv <= 1 + 1e-12)
    else:
        assert np.all(np.sum(ph * ph + pv * pv, axis=0) <= 1 + 1e-12)
    # padded dual entries stay zero
    assert np.all(ph[:, :, -1] == 0) and np.all(pv[:, -1, :] == 0)
    # shift invariance
    np.testing.assert_allclose(O.fgp_prox(x + 0.37, lam, S, tv), th + 0.37, atol=1e-12)
    # flips: ATV is separable, so reversing rows or columns commutes with it.
    # The isotropic forms pair D_h and D_v at the same (i, j), which a flip
    # turns into a different pairing, so they are not flip-equivariant.
    if tv == "atv":
        np.testing.assert_allclose(O.fgp_prox(x[:, ::-1, :], lam, S, tv), th[:, ::-1, :], atol=1e-12)
        np.testing.assert_allclose(O.fgp_prox(x[:, :, ::-1], lam, S, tv), th[:, :, ::-1], atol=1e-12)
    # frame permutation
    perm = [2, 0, 1]
    np.testing.assert_allclose(O.fgp_prox(x[perm], lam, S, tv), th[perm], atol=1e-12)


@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_fgp_transpose_equivariance(tv):
    x = _rand(4, (2, 6, 6))
    th = O.fgp_prox(x, 0.1, 7, tv)
    np.testing.assert_allclose(O.fgp_prox(x.transpose(0, 2, 1), 0.1, 7, tv),
                               th.transpose(0, 2, 1), atol=1e-12)


@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_constant_frames_are_fixed(tv):
    x = np.stack([np.full((5, 4), v) for v in (0.1, 0.5, 0.9)])
    for S in (1, 3, 10):
        th, (ph, pv) = O.fgp_prox(x, 0.05, S, tv, return_dual=True)
        np.testing.assert_array_equal(th, x)
        assert np.all(ph == 0) and np.all(pv == 0)


@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_gradient_projection_dual_objective_monotone(tv):
    """Without momentum (nu = 1) the dual method is gradient projection with
    step 1/L, whose dual objective never decreases."""
    x = _rand(8, (2, 6, 6))
    lam = 0.1
    vals = []
    for S in range(1, 25):
        _, (ph, pv) = O.fgp_prox(x, lam, S, tv, momentum=False, return_dual=True)
        vals.append(O.dual_objective(ph, pv, x, lam))
    assert all(b >= a - 1e-13 for a, b in zip(vals, vals[1:]))


@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_fgp_decreases_primal_objective(tv):
    x = _rand(9, (3, 8, 8))
    lam = 0.05
    f0 = O.prox_objective(x, x, lam, tv)
    for S in (1, 2, 5, 10):
        assert O.prox_objective(O.fgp_prox(x, lam, S, tv), x, lam, tv) < f0
