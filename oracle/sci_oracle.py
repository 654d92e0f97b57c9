"""Plain FP64 oracle for video SCI reconstruction with GAP-TV and ADMM-TV.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the CUDA library.

Follows X. Yuan, "Various Total Variation for Snapshot Video Compressive
Imaging" (arXiv 2005.08028).  Equation numbers count the paper's numbered
displays in order: Eq. 1 (y = Phi x + g), Eq. 2 (Phi = [D_1..D_B]), Eq. 3
(Y = sum X_k . C_k + G), Eq. 4 (per-pixel form), Eq. 5 (x stacking), Eq. 6
(the TV-regularised problem), Eq. 7 (D_h, D_v), Eqs. 8-10 (ATV, ITV2D,
ITV3D), Eqs. 11-13 (the three problems), Eqs. 14-17 (FISTA), Eqs. 18-20
(TwIST), Eqs. 21-22 (GAP), Eqs. 23-26 (ADMM), Eqs. 27-32 (the ITV2D/ITV3D
dual projections); Algorithm 1 is the GAP-ATV-Clip/Cham/FGP listing.

Arrays are ``[B][nx][ny]`` float64: frame k, row i (vertical, D_v), column j
(horizontal, D_h).  Masks are dense arrays of the same shape (any real values;
the synthetic workloads use binary ones).

Readings where the paper is silent or garbled:
  * D_h, D_v are forward differences without wrap-around (Eq. 7 gives
    n-1 rows); duals are padded to full size with zeros in the last column
    (h) / last row (v).
  * ITV2D and ITV3D take the per-pixel Euclidean norm that the projections
    of Eqs. 29-32 imply (Eqs. 9-10 as printed take whole-frame norms).  ITV3D
    ("VTV") couples the B frames of a pixel; no TV has a temporal difference.
  * TVdenoise(x) is the proximal map argmin_t 1/2||t - x||^2 + lam*TV(t): the
    FGP step 1/(8 lam) and t = x - lam*D^T w of Algorithm 1 fix this scale.
  * FGP starts from w = p = 0 and nu = 1 at every TVdenoise call and returns
    t = x - lam*D^T p after S dual updates (Beck & Teboulle's output).  The
    dual warm start (``warm_start=True`` on gap_tv / admm_tv) instead keeps
    the box's w from one call to the next, as Algorithm 1 initialises w once
    before its outer loop, and still resets nu to 1 inside the box; the FGP
    box carries its last momentum point w (which may lie outside the dual
    set), the Chambolle box its w.
  * Loops run exactly T outer and S inner iterations.
  * The Clip box of Algorithm 1 (ATV only) clips at T = lam with step
    1/alpha, alpha = 4, and outputs x - D_h^T w_h - D_v^T w_v from its final
    duals (clip_prox states why).
  * The Chambolle box of Algorithm 1 is read with its D^T as the divergence
    (minus the adjoint), as in Chambolle's derivation; with the adjoint its
    update ascends.  It keeps the max(1, |.|) denominator the paper states it
    used.
  * Pixels with R = sum_k C_k^2 = 0 use the pseudo-inverse (R^+ = 0).
  * ADMM's TVdenoise uses the same lam as GAP (Eq. 25 has no rho).
  * FISTA (Sec. 2.2): L(f) = ||Phi||^2 = max_ij R_ij (Phi Phi^T = diag(R));
    its momentum reads theta^(t+1) = x^(t) + ((tau_t - 1)/tau_{t+1})
    (x^(t) - x^(t-1)) with tau_1 = 1 (the printed update's indices are
    garbled); TVdenoise takes the same lam as GAP (plug-in reading), so its
    fixed points minimise 1/2||y - Phi x||^2 + lam L TV(x).
  * TwIST (Sec. 2.2): its unit step runs on Phi / sqrt(L); alpha and beta
    ("determined by the eigenvalues of Phi^T Phi") follow TwIST's own rule
    with the extreme nonzero eigenvalues of the normalised operator
    (xim = 1, xi1 = min_{R>0} R / max R); the first iteration is a plain
    step; TVdenoise takes lam as for FISTA.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "TV_TYPES", "forward", "adjoint", "mask_energy", "gap_project", "admm_xupdate",
    "grad_h", "grad_v", "grad_h_adj", "grad_v_adj", "div_adj", "tv_value",
    "dual_project", "fgp_momentum_coeffs", "fgp_prox", "divergence", "cham_prox", "CLIP_ALPHA", "clip_prox",
    "prox_objective",
    "dual_objective", "gap_tv", "admm_tv", "lipschitz", "fista_tv", "twist_params", "twist_xi1", "twist_tv",
    "psnr",
    "residual_sq",
]

TV_TYPES = ("atv", "itv2d", "vtv")


# --------------------------------------------------------------------------
# Measurement model (Sec. 1, Eqs. 1-5)
# --------------------------------------------------------------------------

def forward(x: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Phi x: Y = sum_k X_k (.) C_k (Eq. 3 without noise; Eq. 4 per pixel)."""
    x = np.asarray(x, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    return np.sum(x * C, axis=0)


def adjoint(y: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Phi^T y: frame k is C_k (.) Y, since Phi = [D_1 .. D_B] with diagonal D_k (Eq. 2)."""
    y = np.asarray(y, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    return C * y[None, :, :]


def mask_energy(C: np.ndarray) -> np.ndarray:
    """R = diag(Phi Phi^T) = sum_k C_k^2, per pixel (Sec. 2.2, ADMM paragraph)."""
    C = np.asarray(C, dtype=np.float64)
    return np.sum(C * C, axis=0)


def _pinv_diag(d: np.ndarray) -> np.ndarray:
    """Pseudo-inverse of a diagonal: 1/d where d != 0, else 0."""
    out = np.zeros_like(d)
    nz = d != 0
    out[nz] = 1.0 / d[nz]
    return out


def gap_project(theta: np.ndarray, y: np.ndarray, C: np.ndarray) -> np.ndarray:
    """GAP Euclidean projection onto {x : Phi x = y} (Eq. 21; Algorithm 1).

    x = theta + Phi^T (Phi Phi^T)^+ (y - Phi theta), with Phi Phi^T = diag(R).
    """
    theta = np.asarray(theta, dtype=np.float64)
    r = _pinv_diag(mask_energy(C)) * (np.asarray(y, np.float64) - forward(theta, C))
    return theta + adjoint(r, C)


def admm_xupdate(theta: np.ndarray, u: np.ndarray, y: np.ndarray, C: np.ndarray,
                 rho: float) -> np.ndarray:
    """ADMM x-update, Eq. 24: argmin_x 1/2||y - Phi x||^2 + rho/2 ||x - theta + u||^2.

    The normal equations (Phi^T Phi + rho I) x = Phi^T y + rho v with v = theta - u
    are solved in closed form through x = v + Phi^T w, which turns them into
    (Phi Phi^T + rho I) w = y - Phi v: a diagonal system because Phi Phi^T = diag(R).
    At rho = 0 this is the GAP projection of v (pseudo-inverse on R = 0 pixels).
    """
    v = np.asarray(theta, np.float64) - np.asarray(u, np.float64)
    d = mask_energy(C) + rho
    w = _pinv_diag(d) * (np.asarray(y, np.float64) - forward(v, C))
    return v + adjoint(w, C)


# --------------------------------------------------------------------------
# Gradient operators (Eq. 7) and TV (Eqs. 8-10)
# --------------------------------------------------------------------------

def grad_h(x: np.ndarray) -> np.ndarray:
    """D_h applied to every frame: X_k D_h^T, forward difference along j.

    Entry (k, i, j) = x[k, i, j+1] - x[k, i, j] for j < ny-1 and 0 in the last
    column (the n_y - 1 differences of Eq. 7, padded to full size).
    """
    x = np.asarray(x, dtype=np.float64)
    g = np.zeros_like(x)
    g[:, :, :-1] = x[:, :, 1:] - x[:, :, :-1]
    return g


def grad_v(x: np.ndarray) -> np.ndarray:
    """D_v applied to every frame: D_v X_k, forward difference along i (Eq. 7)."""
    x = np.asarray(x, dtype=np.float64)
    g = np.zeros_like(x)
    g[:, :-1, :] = x[:, 1:, :] - x[:, :-1, :]
    return g


def grad_h_adj(w: np.ndarray) -> np.ndarray:
    """D_h^T w for a padded dual (the last column of w is ignored).

    (D_h^T w)[i, j] = w[i, j-1] (if j >= 1) - w[i, j] (if j <= ny-2).
    """
    w = np.asarray(w, dtype=np.float64)
    out = np.zeros_like(w)
    ny = w.shape[2]
    out[:, :, :ny - 1] -= w[:, :, :ny - 1]
    out[:, :, 1:] += w[:, :, :ny - 1]
    return out


def grad_v_adj(w: np.ndarray) -> np.ndarray:
    """D_v^T w for a padded dual (the last row of w is ignored)."""
    w = np.asarray(w, dtype=np.float64)
    out = np.zeros_like(w)
    nx = w.shape[1]
    out[:, :nx - 1, :] -= w[:, :nx - 1, :]
    out[:, 1:, :] += w[:, :nx - 1, :]
    return out


def div_adj(wh: np.ndarray, wv: np.ndarray) -> np.ndarray:
    """D^T w = D_h^T w_h + D_v^T w_v."""
    return grad_h_adj(wh) + grad_v_adj(wv)


def tv_value(x: np.ndarray, tv: str) -> float:
    """TV(x) for 'atv' (Eq. 8), 'itv2d' (Eq. 9) or 'vtv' (= ITV3D, Eq. 10).

    ATV sums |differences|.  ITV2D sums, per frame and pixel,
    sqrt(gh^2 + gv^2).  VTV sums, per pixel, sqrt(sum_k (gh_k^2 + gv_k^2)).
    """
    gh, gv = grad_h(x), grad_v(x)
    if tv == "atv":
        return float(np.sum(np.abs(gh)) + np.sum(np.abs(gv)))
    if tv == "itv2d":
        return float(np.sum(np.sqrt(gh * gh + gv * gv)))
    if tv == "vtv":
        return float(np.sum(np.sqrt(np.sum(gh * gh + gv * gv, axis=0))))
    raise ValueError(f"unknown tv {tv!r}")


# --------------------------------------------------------------------------
# FGP TV proximal map (Sec. 2.3; Algorithm 1, ATV-FGP box; Eqs. 29-32)
# --------------------------------------------------------------------------

def dual_project(ah: np.ndarray, av: np.ndarray, tv: str):
    """Projection of the dual pair onto the unit set of the chosen TV.

    ATV: each entry divided by max(1, |entry|) (Algorithm 1, ATV-FGP box).
    ITV2D: both entries of a voxel divided by max(1, sqrt(ah^2 + av^2))
    (Eqs. 29-30).  VTV: all 2B entries of a pixel divided by
    max(1, sqrt(sum_k ah_k^2 + av_k^2)) (Eqs. 31-32).
    """
    if tv == "atv":
        return ah / np.maximum(1.0, np.abs(ah)), av / np.maximum(1.0, np.abs(av))
    if tv == "itv2d":
        den = np.maximum(1.0, np.sqrt(ah * ah + av * av))
        return ah / den, av / den
    if tv == "vtv":
        den = np.maximum(1.0, np.sqrt(np.sum(ah * ah + av * av, axis=0)))[None]
        return ah / den, av / den
    raise ValueError(f"unknown tv {tv!r}")


def fgp_momentum_coeffs(S: int) -> np.ndarray:
    """(nu_s - 1)/nu_{s+1} for s = 0..S-1, with nu_0 = 1 and
    nu_{s+1} = (1 + sqrt(1 + 4 nu_s^2))/2 (Algorithm 1, ATV-FGP box)."""
    out = np.zeros(S)
    nu = 1.0
    for s in range(S):
        nu_next = (1.0 + np.sqrt(1.0 + 4.0 * nu * nu)) / 2.0
        out[s] = (nu - 1.0) / nu_next
        nu = nu_next
    return out


def fgp_prox(x: np.ndarray, lam: float, S: int, tv: str, *, momentum: bool = True,
             return_dual: bool = False, w0=None, return_state: bool = False):
    """S iterations of FGP for argmin_t 1/2||t - x||^2 + lam*TV(t).

    Per iteration s (Algorithm 1, ATV-FGP box, with Eqs. 29-32 for ITV2D/VTV):
      theta = x - lam (D_h^T w_h + D_v^T w_v)
      a = w + (1/(8 lam)) D theta
      p_new = dual_project(a)
      w = p_new + ((nu_s - 1)/nu_{s+1}) (p_new - p)
    Output theta = x - lam D^T p after the S dual updates.  ``momentum=False``
    gives the plain gradient-projection method (all coefficients 0).

    w starts at 0, or at ``w0 = (w_h, w_v)`` (the dual warm start: Algorithm 1
    sets w once before its outer loop and resets only nu inside the box, so
    nu_0 = 1 still and the first coefficient is 0).  ``return_state=True``
    returns (theta, (w_h, w_v)) with the box's final w, the state a warm
    start carries to the next call; ``return_dual=True`` returns
    (theta, (p_h, p_v)).
    """
    if return_dual and return_state:
        raise ValueError("return_dual and return_state are exclusive")
    x = np.asarray(x, dtype=np.float64)
    step = 1.0 / (8.0 * lam)
    coef = fgp_momentum_coeffs(S) if momentum else np.zeros(S)
    if w0 is None:
        wh = np.zeros_like(x)
        wv = np.zeros_like(x)
    else:
        wh = np.array(w0[0], dtype=np.float64)
        wv = np.array(w0[1], dtype=np.float64)
    ph = np.zeros_like(x)
    pv = np.zeros_like(x)
    for s in range(S):
        theta = x - lam * div_adj(wh, wv)
        ah = wh + step * grad_h(theta)
        av = wv + step * grad_v(theta)
        ph_new, pv_new = dual_project(ah, av, tv)
        wh = ph_new + coef[s] * (ph_new - ph)
        wv = pv_new + coef[s] * (pv_new - pv)
        ph, pv = ph_new, pv_new
    theta = x - lam * div_adj(ph, pv)
    if return_state:
        return theta, (wh, wv)
    if return_dual:
        return theta, (ph, pv)
    return theta


def divergence(wh: np.ndarray, wv: np.ndarray) -> np.ndarray:
    """div w = -(D_h^T w_h + D_v^T w_v): the divergence, minus the adjoint of
    the forward-difference gradient (the reading of D^T in the Chambolle box)."""
    return -div_adj(wh, wv)


def cham_prox(x: np.ndarray, lam: float, S: int, tv: str, *, return_dual: bool = False, w0=None,
              return_state: bool = False):
    """S iterations of Chambolle's dual algorithm for argmin_t 1/2||t - x||^2 + lam*TV(t).

    Algorithm 1, ATV-Cham box (ITV2D-Cham and the ITV3D dual take the norms
    of Eqs. 29-32, as in dual_project), with delta t = 1/8, w = 0 and
    p_d = 0 at the start.  Per iteration s:
      z   = p_d - x / lam
      z_h = D_h z,  z_v = D_v z
      w   = (w + delta t z) / max(1, |w + delta t z|)
      p_d = div w
    Output theta = x - lam p_d.  ``w0 = (w_h, w_v)`` starts from that w
    instead (dual warm start), with p_d = div w0.  ``return_dual`` and
    ``return_state`` both return (theta, (w_h, w_v)): w is this box's whole
    state.
    """
    x = np.asarray(x, dtype=np.float64)
    dt = 1.0 / 8.0
    if w0 is None:
        wh = np.zeros_like(x)
        wv = np.zeros_like(x)
        pd = np.zeros_like(x)
    else:
        wh = np.array(w0[0], dtype=np.float64)
        wv = np.array(w0[1], dtype=np.float64)
        pd = divergence(wh, wv)
    for _ in range(S):
        z = pd - x / lam
        zh, zv = grad_h(z), grad_v(z)
        wh, wv = dual_project(wh + dt * zh, wv + dt * zv, tv)
        pd = divergence(wh, wv)
    theta = x - lam * pd
    if return_dual or return_state:
        return theta, (wh, wv)
    return theta


CLIP_ALPHA = 4.0  # 1/alpha is the clipping step; ||D_h||^2, ||D_v||^2 <= 4 for 1-D differences


def clip_prox(x: np.ndarray, lam: float, S: int, tv: str = "atv", *, alpha: float = CLIP_ALPHA,
              thresh: float | None = None, return_dual: bool = False, w0=None, return_state: bool = False):
    """S iterations of the ATV-Clip box of Algorithm 1 (Selesnick's iterative
    clipping, Sec. 2.3), with unscaled duals w_h, w_v.  Per iteration s:
      theta_h = x - D_h^T w_h,    theta_v = x - D_v^T w_v
      w_h = clip(w_h + (1/alpha) D_h theta_h, T),  w_v likewise with D_v, theta_v
    where clip(a, T) = min(max(a, -T), T).  Output theta_h + theta_v - x,
    formed from the final w: x - D_h^T w_h - D_v^T w_v.

    Readings (the box leaves alpha undefined and prints the threshold 2 lam):
    T = lam, so that a converged box gives, per direction, the exact 1-D
    proximal map of lam * TV -- the same scale as the FGP and Chambolle boxes
    (prox of lam TV under 1/2||theta - x||^2; the printed 2 lam matches a
    fidelity without the 1/2); alpha = 4, the bound on the largest eigenvalue
    of D_h D_h^T (and D_v D_v^T), which makes the clipped step converge; the
    output uses the duals after the S-th update, as for FGP (Beck and
    Teboulle's output).  The two directions never interact inside the box:
    on a frame constant along one axis it is that axis's exact 1-D TV prox;
    in general the output is x minus the sum of the two 1-D corrections.

    ``w0 = (w_h, w_v)`` starts from those duals (the dual warm start);
    ``return_dual`` / ``return_state`` return (theta, (w_h, w_v))."""
    if tv != "atv":
        raise ValueError("the Clip box is an ATV solver")
    x = np.asarray(x, dtype=np.float64)
    T = lam if thresh is None else float(thresh)
    if w0 is None:
        wh = np.zeros_like(x)
        wv = np.zeros_like(x)
    else:
        wh = np.array(w0[0], dtype=np.float64)
        wv = np.array(w0[1], dtype=np.float64)
    for _ in range(S):
        th_h = x - grad_h_adj(wh)
        th_v = x - grad_v_adj(wv)
        wh = np.clip(wh + grad_h(th_h) / alpha, -T, T)
        wv = np.clip(wv + grad_v(th_v) / alpha, -T, T)
    theta = x - grad_h_adj(wh) - grad_v_adj(wv)
    if return_dual or return_state:
        return theta, (wh, wv)
    return theta


def _tv_denoise(dual: str):
    """TVdenoise of Algorithm 1: the FGP, Chambolle or Clip box."""
    if dual == "fgp":
        return fgp_prox
    if dual == "cham":
        return cham_prox
    if dual == "clip":
        return clip_prox
    raise ValueError(f"unknown dual solver {dual!r}")


def prox_objective(theta: np.ndarray, x: np.ndarray, lam: float, tv: str) -> float:
    """Primal objective 1/2||theta - x||^2 + lam*TV(theta)."""
    d = np.asarray(theta, np.float64) - np.asarray(x, np.float64)
    return 0.5 * float(np.sum(d * d)) + lam * tv_value(theta, tv)


def dual_objective(ph: np.ndarray, pv: np.ndarray, x: np.ndarray, lam: float) -> float:
    """Dual objective 1/2||x||^2 - 1/2||x - lam D^T p||^2 for a feasible p.

    For every feasible p it is at most the primal optimum, so the primal
    minus this value bounds the suboptimality of theta = x - lam D^T p.
    """
    x = np.asarray(x, np.float64)
    t = x - lam * div_adj(ph, pv)
    return 0.5 * float(np.sum(x * x)) - 0.5 * float(np.sum(t * t))


# --------------------------------------------------------------------------
# Outer frameworks (Sec. 2.2; Algorithm 1)
# --------------------------------------------------------------------------

def gap_tv(y: np.ndarray, C: np.ndarray, lam: float, T: int, S: int, tv: str,
           theta0: np.ndarray | None = None, dual: str = "fgp", warm_start: bool = False):
    """GAP-TV (Eqs. 21-22; Algorithm 1): returns (x^(T), theta^(T)).

    theta^(0) = Phi^T y unless ``theta0`` is given (resuming).  Each of the T
    iterations projects onto {Phi x = y} and applies the S-step TVdenoise
    (``dual`` = 'fgp', 'cham' or 'clip': the FGP, Chambolle or Clip box).
    ``warm_start=True`` carries the box's w from each TVdenoise call to the
    next (Algorithm 1 initialises w once, before the outer loop); w starts at
    0 in the first call.
    """
    denoise = _tv_denoise(dual)
    theta = adjoint(y, C) if theta0 is None else np.array(theta0, dtype=np.float64)
    x = theta
    w = None
    for _ in range(T):
        x = gap_project(theta, y, C)
        if warm_start:
            theta, w = denoise(x, lam, S, tv, w0=w, return_state=True)
        else:
            theta = denoise(x, lam, S, tv)
    return x, theta


def admm_tv(y: np.ndarray, C: np.ndarray, lam: float, rho: float, T: int, S: int,
            tv: str, theta0: np.ndarray | None = None, u0: np.ndarray | None = None, dual: str = "fgp",
            warm_start: bool = False):
    """ADMM-TV (Eqs. 24-26): returns (x^(T), theta^(T), u^(T)).

    theta^(0) = Phi^T y and u^(0) = 0 unless given.  Per iteration:
    x = admm_xupdate(theta, u), theta = TVdenoise(u + x), u = u + x - theta.
    ``warm_start`` as in gap_tv.
    """
    denoise = _tv_denoise(dual)
    theta = adjoint(y, C) if theta0 is None else np.array(theta0, dtype=np.float64)
    u = np.zeros_like(theta) if u0 is None else np.array(u0, dtype=np.float64)
    x = theta
    w = None
    for _ in range(T):
        x = admm_xupdate(theta, u, y, C, rho)
        if warm_start:
            theta, w = denoise(u + x, lam, S, tv, w0=w, return_state=True)
        else:
            theta = denoise(u + x, lam, S, tv)
        u = u + x - theta
    return x, theta, u


def lipschitz(C: np.ndarray) -> float:
    """L(f) for f(x) = 1/2||y - Phi x||^2: ||Phi||^2 = ||Phi Phi^T|| = max_ij R_ij."""
    return float(np.max(mask_energy(C)))


def fista_tv(y: np.ndarray, C: np.ndarray, lam: float, T: int, S: int, tv: str,
             theta0: np.ndarray | None = None, dual: str = "fgp"):
    """FISTA-TV (Sec. 2.2, FISTA steps): returns (x^(T), x^(T)).

    theta^(1) = Phi^T y unless ``theta0`` is given; tau_1 = 1.  Iteration t:
      z^(t)        = theta^(t) + (1/L) Phi^T (y - Phi theta^(t))
      x^(t)        = TVdenoise(z^(t))
      tau_{t+1}    = (1 + sqrt(1 + 4 tau_t^2)) / 2
      theta^(t+1)  = x^(t) + ((tau_t - 1)/tau_{t+1}) (x^(t) - x^(t-1))
    The estimate is x^(T); it is also returned as the second value, in the
    place where gap_tv returns theta.
    """
    denoise = _tv_denoise(dual)
    L = lipschitz(C)
    step = 0.0 if L == 0.0 else 1.0 / L
    theta = adjoint(y, C) if theta0 is None else np.array(theta0, dtype=np.float64)
    x_prev = np.zeros_like(theta)
    x = theta
    tau = 1.0
    for _ in range(T):
        z = theta + step * adjoint(y - forward(theta, C), C)
        x = denoise(z, lam, S, tv)
        tau_next = (1.0 + np.sqrt(1.0 + 4.0 * tau * tau)) / 2.0
        theta = x + ((tau - 1.0) / tau_next) * (x - x_prev)
        x_prev = x
        tau = tau_next
    return x, x


def twist_params(xi1: float = 1e-4, xim: float = 1.0) -> tuple[float, float]:
    """TwIST's (alpha, beta) for the eigenvalue bounds xi1 <= eig(A^T A) <= xim
    of its (normalised) operator A (Sec. 2.2, TwIST steps, citing
    Bioucas-Dias & Figueiredo 2007, whose rule this is):
      kappa = xi1 / xim,  rho = (1 - sqrt(kappa)) / (1 + sqrt(kappa)),
      alpha = 1 + rho^2,  beta = 2 alpha / (xim + xi1).
    These give the two-step iteration its best worst-case linear rate, rho,
    over the interval.  kappa = 1 gives alpha = beta = 1 (plain IST)."""
    if not (0.0 < xi1 <= xim):
        raise ValueError("need 0 < xi1 <= xim")
    r = np.sqrt(xi1 / xim)
    rho = (1.0 - r) / (1.0 + r)
    alpha = 1.0 + rho * rho
    return alpha, 2.0 * alpha / (xim + xi1)


def twist_xi1(C: np.ndarray) -> float:
    """Smallest nonzero eigenvalue of A^T A for A = Phi / sqrt(L): the
    eigenvalues of Phi^T Phi are 0 (its nullspace) and the R_ij, so this is
    min_{R > 0} R / max R (1 when nothing is measured)."""
    R = mask_energy(C)
    pos = R[R > 0]
    return 1.0 if pos.size == 0 else float(pos.min() / pos.max())


def twist_tv(y: np.ndarray, C: np.ndarray, lam: float, T: int, S: int, tv: str,
             theta0: np.ndarray | None = None, dual: str = "fgp", xi1: float | None = None):
    """TwIST-TV (Sec. 2.2, TwIST steps): returns (x^(T), theta^(T-1)).

    The printed steps take a unit gradient step, which needs ||Phi|| <= 1;
    they run here on A = Phi / sqrt(L) and y / sqrt(L) (L = max R, as for
    FISTA), so the step reads z = x + (1/L) Phi^T (y - Phi x).  alpha and
    beta come from the eigenvalues of A^T A (twist_params with xim = 1 and
    xi1 = twist_xi1(C), its smallest nonzero eigenvalue; the nullspace is
    left to the TV term).  ``xi1`` overrides it (TwIST's authors use 1e-4
    for ill-conditioned operators, with a monotone safeguard that the
    printed steps do not have).  x^(0) = Phi^T y
    unless ``theta0`` is given; the first iteration is one plain step
    x^(1) = theta^(0) (TwIST starts its two-step recursion from an IST step),
    then for t >= 1:
      z^(t)       = x^(t) + (1/L) Phi^T (y - Phi x^(t))
      theta^(t)   = TVdenoise(z^(t))
      x^(t+1)     = (1 - alpha) x^(t-1) + (alpha - beta) x^(t) + beta theta^(t)
    TVdenoise takes lam as for FISTA, so fixed points minimise
    1/2||y - Phi x||^2 + lam L TV(x).  theta^(T-1) is x^(0) when T = 0.
    """
    denoise = _tv_denoise(dual)
    L = lipschitz(C)
    step = 0.0 if L == 0.0 else 1.0 / L
    alpha, beta = twist_params(twist_xi1(C) if xi1 is None else xi1, 1.0)
    x = adjoint(y, C) if theta0 is None else np.array(theta0, dtype=np.float64)
    x_prev = x
    theta = x
    for t in range(T):
        z = x + step * adjoint(y - forward(x, C), C)
        theta = denoise(z, lam, S, tv)
        if t == 0:
            x_next = theta
        else:
            x_next = (1.0 - alpha) * x_prev + (alpha - beta) * x + beta * theta
        x_prev, x = x, x_next
    return x, theta


# --------------------------------------------------------------------------
# Metrics (the paper reports PSNR, Table 1; its definition is not stated)
# --------------------------------------------------------------------------

def psnr(x: np.ndarray, ref: np.ndarray, peak: float = 1.0) -> float:
    """10 log10(peak^2 / MSE) with the MSE over the whole cube, no clipping."""
    d = np.asarray(x, np.float64) - np.asarray(ref, np.float64)
    mse = float(np.mean(d * d))
    return float("inf") if mse == 0.0 else 10.0 * np.log10(peak * peak / mse)


def residual_sq(theta: np.ndarray, y: np.ndarray, C: np.ndarray) -> float:
    """||y - Phi theta||_2^2."""
    r = np.asarray(y, np.float64) - forward(theta, C)
    return float(np.sum(r * r))
