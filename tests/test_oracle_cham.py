"""Pins for the oracle's Chambolle TVdenoise (Algorithm 1, ATV-Cham box;
ITV2D-Cham and the ITV3D dual with the norms of Eqs. 29-32).

The printed box is read with its D^T as the divergence (minus the adjoint).
The pins:
- that reading is the projected dual gradient step, i.e. FGP with nu = 1,
  a separately written function;
- the literal reading (D^T as the adjoint) ends worse than doing nothing;
- converged iterates match an independent SciPy solve of the dual problem;
- the dual objective never decreases (projected gradient with step 1/8 <= 1/L);
- constant frames are fixed points;
- GAP-TV built on it still lands on {Phi x = y}.
"""
import numpy as np
import pytest

import oracle as O
from test_oracle_prox import _dual_solve_scipy


def _rand(seed, shape):
    return np.random.default_rng(seed).random(shape)


@pytest.mark.parametrize("tv", O.TV_TYPES)
@pytest.mark.parametrize("S", [1, 2, 7, 40])
def test_divergence_reading_is_gradient_projection(tv, S):
    x = _rand(S + 3, (3, 7, 6))
    for lam in (0.05, 0.3):
        a = O.cham_prox(x, lam, S, tv)
        b = O.fgp_prox(x, lam, S, tv, momentum=False)
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)


@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_literal_adjoint_reading_ascends(tv):
    """With D^T read as the adjoint the printed update moves away from the
    minimiser: its output is worse than x itself, the divergence reading's
    is better."""
    x = _rand(3, (2, 6, 6))
    lam = 0.1
    wh, wv, pd = np.zeros_like(x), np.zeros_like(x), np.zeros_like(x)
    for _ in range(50):
        z = pd - x / lam
        wh, wv = O.dual_project(wh + O.grad_h(z) / 8, wv + O.grad_v(z) / 8, tv)
        pd = O.div_adj(wh, wv)
    f_x = O.prox_objective(x, x, lam, tv)
    assert O.prox_objective(x - lam * pd, x, lam, tv) > f_x
    assert O.prox_objective(O.cham_prox(x, lam, 50, tv), x, lam, tv) < f_x


@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_converged_cham_matches_scipy_dual_solve(tv):
    x = _rand({"atv": 21, "itv2d": 22, "vtv": 23}[tv], (2, 4, 4))
    lam = 0.05
    th = O.cham_prox(x, lam, 20000, tv)
    ref = _dual_solve_scipy(x, lam, tv)
    np.testing.assert_allclose(th, ref, atol=2e-5)


@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_cham_dual_objective_never_decreases(tv):
    x = _rand(31, (2, 6, 6))
    lam = 0.1
    vals = []
    for S in range(1, 30):
        _, (wh, wv) = O.cham_prox(x, lam, S, tv, return_dual=True)
        # the box's w is minus the dual variable of theta = x - lam D^T p
        vals.append(O.dual_objective(-wh, -wv, x, lam))
    assert all(b >= a - 1e-13 for a, b in zip(vals, vals[1:]))


@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_cham_constant_frames_are_fixed(tv):
    x = np.broadcast_to(np.arange(3.0)[:, None, None] * 0.3, (3, 5, 4)).copy()
    th, (wh, wv) = O.cham_prox(x, 0.2, 10, tv, return_dual=True)
    np.testing.assert_array_equal(th, x)
    assert np.all(wh == 0) and np.all(wv == 0)


@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_gap_cham_output_is_feasible(tv):
    rng = np.random.default_rng(41)
    C = (rng.random((4, 9, 8)) < 0.5).astype(np.float64)
    y = O.forward(rng.random((4, 9, 8)), C)
    x, th = O.gap_tv(y, C, 0.05, 5, 4, tv, dual="cham")
    covered = O.mask_energy(C) > 0
    np.testing.assert_allclose(O.forward(x, C)[covered], y[covered], atol=1e-12)
    # and it differs from the FGP-based solve (the box is not a no-op switch)
    _, th_fgp = O.gap_tv(y, C, 0.05, 5, 4, tv)
    assert np.max(np.abs(th - th_fgp)) > 1e-6
