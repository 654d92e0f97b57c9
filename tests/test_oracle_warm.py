"""Pins of the oracle's dual warm start (Algorithm 1 initialises the box's w
once, before the outer loop, and resets only nu inside the FGP box).

- A warm start from an optimal dual stays optimal: the projected dual step
  has every optimal w as a fixed point, so one update from SciPy's w*
  (an independent solve) returns theta* (FGP; the Chambolle box, whose w is
  minus FGP's, from -w*).  A cold start is far from it after one update.
- Splitting a momentum-free run (the Chambolle box; FGP without momentum)
  into S1 + S2 updates with the state carried equals one run of S1 + S2
  updates bit for bit: the carried w is the box's whole state.
- With one outer iteration the warm start changes nothing (w starts at 0).
- With converged TVdenoise calls, warm- and cold-started GAP-TV / ADMM-TV
  agree: the prox is unique, whatever dual it starts from.
"""
import numpy as np
import pytest

import oracle as O
import sci_synth as ss
from test_oracle_prox import _dual_solve_scipy


def _rand(seed, shape):
    return np.random.default_rng(seed).random(shape)


@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_one_update_from_an_optimal_dual_returns_the_prox(tv):
    x = _rand({"atv": 31, "itv2d": 32, "vtv": 33}[tv], (2, 4, 4))
    lam = 0.05
    th_star, (wh, wv) = _dual_solve_scipy(x, lam, tv, return_w=True)
    cold = O.fgp_prox(x, lam, 1, tv)
    assert np.abs(cold - th_star).max() > 1e-3
    for S in (1, 4):
        np.testing.assert_allclose(O.fgp_prox(x, lam, S, tv, w0=(wh, wv)), th_star, atol=1e-7)
        np.testing.assert_allclose(O.cham_prox(x, lam, S, tv, w0=(-wh, -wv)), th_star, atol=1e-7)
    # the FGP box's state after such a start is still optimal
    _, (sh, sv) = O.fgp_prox(x, lam, 3, tv, w0=(wh, wv), return_state=True)
    np.testing.assert_allclose(x - lam * O.div_adj(sh, sv), th_star, atol=1e-7)


@pytest.mark.parametrize("tv", O.TV_TYPES)
@pytest.mark.parametrize("S1,S2", [(1, 1), (3, 5), (7, 2)])
def test_momentum_free_runs_split_exactly(tv, S1, S2):
    x = _rand(40 + S1 + 10 * S2, (3, 5, 6))
    lam = 0.08
    _, w = O.cham_prox(x, lam, S1, tv, return_state=True)
    np.testing.assert_array_equal(O.cham_prox(x, lam, S2, tv, w0=w), O.cham_prox(x, lam, S1 + S2, tv))
    _, w = O.fgp_prox(x, lam, S1, tv, momentum=False, return_state=True)
    np.testing.assert_array_equal(O.fgp_prox(x, lam, S2, tv, momentum=False, w0=w),
                                  O.fgp_prox(x, lam, S1 + S2, tv, momentum=False))


def test_fgp_state_is_the_last_momentum_point():
    x = _rand(50, (2, 5, 5))
    lam, S = 0.05, 4
    _, (ph, pv) = O.fgp_prox(x, lam, S, "itv2d", return_dual=True)
    _, (ph1, pv1) = O.fgp_prox(x, lam, S - 1, "itv2d", return_dual=True)
    _, (wh, wv) = O.fgp_prox(x, lam, S, "itv2d", return_state=True)
    c = O.fgp_momentum_coeffs(S)[S - 1]
    assert c > 0
    np.testing.assert_allclose(wh, ph + c * (ph - ph1), atol=1e-15)
    np.testing.assert_allclose(wv, pv + c * (pv - pv1), atol=1e-15)
    with pytest.raises(ValueError):
        O.fgp_prox(x, lam, S, "itv2d", return_dual=True, return_state=True)


@pytest.mark.parametrize("dual", ["fgp", "cham"])
@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_one_outer_iteration_is_unchanged(dual, tv):
    case = ss.make_case(7, 9, 4, 60, sigma=0.01)
    y = O.forward(case.x_gt, case.masks) + case.noise
    a = O.gap_tv(y, case.masks, 0.05, 1, 6, tv, dual=dual)
    b = O.gap_tv(y, case.masks, 0.05, 1, 6, tv, dual=dual, warm_start=True)
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)
    a = O.admm_tv(y, case.masks, 0.05, 0.01, 1, 6, tv, dual=dual)
    b = O.admm_tv(y, case.masks, 0.05, 0.01, 1, 6, tv, dual=dual, warm_start=True)
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)


@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_warm_start_changes_later_iterations(tv):
    case = ss.make_case(7, 9, 4, 61, sigma=0.01)
    y = O.forward(case.x_gt, case.masks) + case.noise
    xa, _ = O.gap_tv(y, case.masks, 0.05, 3, 2, tv)
    xb, _ = O.gap_tv(y, case.masks, 0.05, 3, 2, tv, warm_start=True)
    assert np.abs(xa - xb).max() > 1e-6


@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_converged_warm_and_cold_loops_agree(tv):
    case = ss.make_case(6, 5, 3, 7, sigma=0.0)
    y = O.forward(case.x_gt, case.masks)
    xc, tc = O.gap_tv(y, case.masks, 0.1, 3, 2000, tv)
    xw, tw = O.gap_tv(y, case.masks, 0.1, 3, 2000, tv, warm_start=True)
    np.testing.assert_allclose(xw, xc, atol=1e-6)
    np.testing.assert_allclose(tw, tc, atol=1e-6)
    xc, tc, uc = O.admm_tv(y, case.masks, 0.1, 0.01, 3, 2000, tv)
    xw, tw, uw = O.admm_tv(y, case.masks, 0.1, 0.01, 3, 2000, tv, warm_start=True)
    np.testing.assert_allclose(tw, tc, atol=1e-6)
    np.testing.assert_allclose(uw, uc, atol=1e-6)
