"""Thin ctypes binding of libsci (include/sci.h) with torch tensors as buffers.

Argument marshalling only: every step of the reconstruction runs in the CUDA
kernels of libsci.so.  torch supplies device memory and the current stream.
If the library cannot be loaded, every call raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

__all__ = [
    "SciError", "TV", "DTYPE", "DUAL", "load", "sci_masks_pack", "sci_forward", "sci_adjoint",
    "sci_project", "sci_tv_prox", "sci_gap_tv", "sci_admm_tv", "sci_fista_tv", "sci_twist_tv", "sci_sqdiff_f64",
    "sci_residual_f64", "sci_graph_cache_clear", "sci_tv_prox_noalloc", "sci_last_solve_launches", "sci_fused_updates", "Batch", "SciProblem",
    "sci_gap_tv_batched", "sci_last_batch_launches", "ALGO", "sci_tune_fuse", "sci_tune_fuse_batched",
    "sci_tune_launch", "sci_tile_classes", "sci_fused_updates_tile",
    "sci_conv3d_c32_bf16", "LearnedProx", "sci_gap_tv_lprox", "Workspace", "SciParams",
]

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsci.so")
_lib = None
_lock = threading.Lock()

TV = {"atv": 0, "itv2d": 1, "vtv": 2}
DTYPE = {"f32": 0, "bf16": 1, "f16": 2}
_STATUS = {0: "SCI_OK", 1: "SCI_ERR_ARG", 2: "SCI_ERR_SHAPE", 3: "SCI_ERR_CUDA",
           4: "SCI_ERR_NONFINITE", 5: "SCI_ERR_TIMEOUT", 6: "SCI_ERR_WORKSPACE"}


class SciError(RuntimeError):
    def __init__(self, fn: str, status: int):
        super().__init__(f"{fn} failed: {_STATUS.get(status, status)}")
        self.status = status


class SciParams(C.Structure):
    _fields_ = [("tv", C.c_int), ("lam", C.c_float), ("rho", C.c_float),
                ("outer_iters", C.c_int), ("inner_iters", C.c_int), ("storage", C.c_int),
                ("fuse_k", C.c_int), ("init", C.c_int), ("use_graph", C.c_int), ("dual", C.c_int),
                ("warm_start", C.c_int), ("check_input", C.c_int), ("tile", C.c_int)]


class SciProblem(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("B", C.c_int), ("y", C.c_void_p), ("bits", C.c_void_p),
                ("theta", C.c_void_p), ("x_out", C.c_void_p)]


_vp, _i, _f, _sz = C.c_void_p, C.c_int, C.c_float, C.c_size_t
_SIGS = {
    "sci_status_str": (C.c_char_p, [_i]),
    "sci_version": (_i, []),
    "sci_masks_pack": (_i, [_vp, _i, _i, _i, _vp, _vp, _vp]),
    "sci_forward": (_i, [_vp, _vp, _i, _i, _i, _vp, _vp]),
    "sci_adjoint": (_i, [_vp, _vp, _i, _i, _i, _vp, _vp]),
    "sci_project": (_i, [_vp, _vp, _vp, _vp, _i, _i, _i, _f, _vp, _vp]),
    "sci_tv_prox_workspace": (_sz, [_i, _i, _i, _i]),
    "sci_tv_prox": (_i, [_vp, _i, _i, _i, _i, _f, _i, _vp, _vp, _sz, _vp]),
    "sci_tv_prox_cham": (_i, [_vp, _i, _i, _i, _i, _f, _i, _vp, _vp, _sz, _vp]),
    "sci_tv_prox_clip": (_i, [_vp, _i, _i, _i, _i, _f, _i, _vp, _vp, _sz, _vp]),
    "sci_solver_workspace": (_sz, [_i, _i, _i, C.POINTER(SciParams)]),
    "sci_gap_tv": (_i, [_vp, _vp, _i, _i, _i, C.POINTER(SciParams), _vp, _vp, _vp, _i, _vp, _sz, _vp]),
    "sci_fista_tv": (_i, [_vp, _vp, _i, _i, _i, C.POINTER(SciParams), _vp, _vp, _vp, _i, _vp, _sz, _vp]),
    "sci_twist_tv": (_i, [_vp, _vp, _i, _i, _i, C.POINTER(SciParams), _vp, _vp, _vp, _i, _vp, _sz, _vp]),
    "sci_admm_tv": (_i, [_vp, _vp, _i, _i, _i, C.POINTER(SciParams), _vp, _vp, _vp, _vp, _i, _vp, _sz,
                         _vp]),
    "sci_graph_cache_clear": (None, []),
    "sci_reduce_workspace": (_sz, []),
    "sci_sqdiff_f64": (_i, [_vp, _vp, _sz, _vp, _vp, _sz, _vp]),
    "sci_residual_f64": (_i, [_vp, _vp, _vp, _i, _i, _i, _vp, _vp, _sz, _vp]),
    "sci_tv_prox_noalloc": (_i, [_vp, _i, _i, _i, _i, _f, _i, _vp, _vp]),
    "sci_tv_prox_noalloc_max_voxels": (C.c_longlong, []),
    "sci_last_solve_launches": (C.c_longlong, []),
    "sci_fused_updates": (_i, [_i, _i, _i, _i]),
    "sci_fused_updates_tile": (_i, [_i, _i, _i, _i, _i]),
    "sci_tile_classes": (_i, [_i, _i, C.POINTER(C.c_int), _i]),
    "sci_tune_launch": (_i, [_i, _vp, _vp, _i, _i, _i, C.POINTER(SciParams), _vp, _vp, _vp, _sz,
                             C.POINTER(C.c_int), C.POINTER(C.c_int), _i, _i, _i, C.POINTER(C.c_float),
                             C.POINTER(C.c_int), _vp]),
    "sci_tune_fuse": (_i, [_i, _vp, _vp, _i, _i, _i, C.POINTER(SciParams), _vp, _vp, _vp, _sz,
                           C.POINTER(_i), _i, _i, _i, C.POINTER(_f), C.POINTER(_i), _vp]),
    "sci_tune_fuse_batched": (_i, [C.POINTER(SciProblem), _i, C.POINTER(SciParams), _vp, _sz,
                                   C.POINTER(_i), _i, _i, _i, C.POINTER(_f), C.POINTER(_i), _vp]),
    "sci_gap_tv_batched_workspace": (_sz, [C.POINTER(SciProblem), _i, C.POINTER(SciParams)]),
    "sci_gap_tv_batched": (_i, [C.POINTER(SciProblem), _i, C.POINTER(SciParams), _vp, _sz, _vp]),
    "sci_last_batch_launches": (C.c_longlong, []),
    "sci_batch_graph_cache_clear": (None, []),
    "sci_lprox_param_count": (_sz, []),
    "sci_lprox_workspace": (_sz, [_i, _i, _i, _i, _i]),
    "sci_lprox_apply": (_i, [_vp, _vp, _i, _i, _i, _i, _vp, _vp, _sz, _vp]),
    "sci_lprox_train_step": (_i, [_vp, _vp, _vp, _i, _f, _vp, _vp, _i, _i, _i, _i, _vp, _vp, _sz, _vp]),
    "sci_lprox_grads": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _vp, _vp, _vp, _sz, _vp]),
    "sci_lprox_error_word": (_i, [_vp, _sz, _i, _i, _i, _i, _i, C.POINTER(C.c_void_p)]),
    "sci_conv3d_c32_bf16": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _i, _vp, _vp, _vp]),
    "sci_gap_tv_lprox_workspace": (_sz, [_i, _i, _i, _i, C.POINTER(SciParams)]),
    "sci_gap_tv_lprox": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _vp, _vp, _i, _vp, _f,
                              C.POINTER(SciParams), _vp, _vp, _vp, _sz, _vp]),
}


def load(path: str | None = None):
    """Load libsci.so (once) and declare the C signatures."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or _LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(
                    f"libsci.so not found at {p}: build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'`")
            lib = C.CDLL(p)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(fn: str, status: int):
    if status != 0:
        raise SciError(fn, status)


def _ptr(t: torch.Tensor | None):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(device: torch.device):
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _need_cuda(*ts):
    for t in ts:
        if t is not None:
            if not t.is_cuda:
                raise ValueError("libsci works on CUDA tensors only")
            if not t.is_contiguous():
                raise ValueError("tensors must be contiguous")


class Workspace:
    """A growable device scratch buffer (torch-allocated, 512-byte aligned)."""

    def __init__(self, device="cuda"):
        self.device = torch.device(device)
        self.buf = None

    def get(self, nbytes: int) -> torch.Tensor:
        nbytes = max(int(nbytes), 256)
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        return self.buf


# ---------------------------------------------------------------- measurement model

def sci_masks_pack(masks: torch.Tensor, check: bool = True) -> torch.Tensor:
    """Dense binary masks uint8 [B][nx][ny] -> packed int32 [nx][ny] (bit k = mask k)."""
    _need_cuda(masks)
    if masks.dtype != torch.uint8 or masks.dim() != 3:
        raise ValueError("masks must be uint8 [B][nx][ny]")
    B, nx, ny = masks.shape
    bits = torch.empty((nx, ny), dtype=torch.int32, device=masks.device)
    bad = torch.zeros(1, dtype=torch.int32, device=masks.device) if check else None
    _check("sci_masks_pack", load().sci_masks_pack(_ptr(masks), nx, ny, B, _ptr(bits), _ptr(bad),
                                                   _stream(masks.device)))
    if check and int(bad.item()) != 0:
        raise ValueError(f"masks must be binary: {int(bad.item())} entries are neither 0 nor 1")
    return bits


def sci_forward(x: torch.Tensor, bits: torch.Tensor) -> torch.Tensor:
    """y = Phi x = sum_k C_k . X_k (Eq. 3)."""
    _need_cuda(x, bits)
    B, nx, ny = x.shape
    y = torch.empty((nx, ny), dtype=torch.float32, device=x.device)
    _check("sci_forward", load().sci_forward(_ptr(x), _ptr(bits), nx, ny, B, _ptr(y), _stream(x.device)))
    return y


def sci_adjoint(y: torch.Tensor, bits: torch.Tensor, B: int) -> torch.Tensor:
    """x = Phi^T y, frame k = C_k . Y (Eq. 2)."""
    _need_cuda(y, bits)
    nx, ny = y.shape
    x = torch.empty((B, nx, ny), dtype=torch.float32, device=y.device)
    _check("sci_adjoint", load().sci_adjoint(_ptr(y), _ptr(bits), nx, ny, B, _ptr(x), _stream(y.device)))
    return x


def sci_project(theta: torch.Tensor, y: torch.Tensor, bits: torch.Tensor, rho: float = 0.0,
                u: torch.Tensor | None = None) -> torch.Tensor:
    """GAP projection (rho = 0, Eq. 21) or ADMM x-update (rho > 0, Eq. 24)."""
    _need_cuda(theta, y, bits, u)
    B, nx, ny = theta.shape
    x = torch.empty_like(theta)
    _check("sci_project", load().sci_project(_ptr(theta), _ptr(u), _ptr(y), _ptr(bits), nx, ny, B,
                                             float(rho), _ptr(x), _stream(theta.device)))
    return x


def sci_tv_prox(x: torch.Tensor, tv: str, lam: float, inner_iters: int,
                work: Workspace | None = None, dual: str = "fgp") -> torch.Tensor:
    """TV proximal map with `inner_iters` dual updates: dual='fgp' (Algorithm 1,
    FGP box; sci_tv_prox), 'cham' (Chambolle box; sci_tv_prox_cham) or 'clip'
    (ATV-Clip box, tv='atv'; sci_tv_prox_clip)."""
    _need_cuda(x)
    B, nx, ny = x.shape
    lib = load()
    need = lib.sci_tv_prox_workspace(nx, ny, B, TV[tv])
    wbuf = (work or Workspace(x.device)).get(need)
    theta = torch.empty_like(x)
    name = {"fgp": "sci_tv_prox", "cham": "sci_tv_prox_cham", "clip": "sci_tv_prox_clip"}[dual]
    _check(name, getattr(lib, name)(_ptr(x), nx, ny, B, TV[tv], float(lam), int(inner_iters),
                                    _ptr(theta), _ptr(wbuf), wbuf.numel(), _stream(x.device)))
    return theta


def sci_tv_prox_noalloc(x: torch.Tensor, tv: str, lam: float, inner_iters: int) -> torch.Tensor:
    """sci_tv_prox with the library's fixed internal scratch (no workspace).

    For callers that cannot allocate device memory; B*nx*ny is limited to
    sci_tv_prox_noalloc_max_voxels().  Concurrent calls on different streams
    race on the shared scratch.
    """
    _need_cuda(x)
    B, nx, ny = x.shape
    theta = torch.empty_like(x)
    _check("sci_tv_prox_noalloc", load().sci_tv_prox_noalloc(_ptr(x), nx, ny, B, TV[tv], float(lam),
                                                             int(inner_iters), _ptr(theta),
                                                             _stream(x.device)))
    return theta


DUAL = {"fgp": 0, "cham": 1, "clip": 2}


def _params(tv, lam, rho, outer, inner, storage, fuse_k, init, use_graph, dual="fgp", warm_start=False,
            check_input=False, tile=0):
    return SciParams(TV[tv], float(lam), float(rho), int(outer), int(inner), DTYPE[storage],
                     int(fuse_k), int(init), int(use_graph), DUAL[dual], int(bool(warm_start)),
                     int(bool(check_input)), int(tile))


def _solve(admm: bool, y, bits, B, tv, lam, outer, inner, rho=0.0, storage="f32", theta=None, u=None, fista=False,
           twist=False,
           init=None, x_out=None, resid=None, resid_every=0, fuse_k=0, use_graph=True, work=None, dual="fgp",
           warm_start=False, check_input=False, tile=0):
    _need_cuda(y, bits, theta, u, x_out, resid)
    nx, ny = y.shape
    dev = y.device
    if init is None:
        init = theta is None
    if theta is None:
        theta = torch.empty((B, nx, ny), dtype=torch.float32, device=dev)
    if admm and u is None:
        if not init:
            raise ValueError("resuming ADMM needs u")
        u = torch.empty((B, nx, ny), dtype=torch.float32, device=dev)
    if x_out is None:
        x_out = torch.empty((B, nx, ny), dtype=torch.float32, device=dev)
    if fuse_k == "tuned":
        from . import tune
        if twist:
            raise ValueError("fuse_k='tuned' covers GAP, ADMM and FISTA; pass a depth for TwIST")
        fuse_k, tile = tune.tuned_launch("admm" if admm else ("fista" if fista else "gap"), y, bits, B, tv, lam,
                                         inner, rho=rho, storage=storage, dual=dual, work=work)
    prm = _params(tv, lam, rho, outer, inner, storage, fuse_k, init, use_graph, dual, warm_start, check_input,
                  tile)
    lib = load()
    need = lib.sci_solver_workspace(nx, ny, B, C.byref(prm))
    wbuf = (work or Workspace(dev)).get(need)
    if resid_every and resid is None:
        resid = torch.zeros(max(1, outer // resid_every), dtype=torch.float64, device=dev)
    if admm:
        st = lib.sci_admm_tv(_ptr(y), _ptr(bits), nx, ny, B, C.byref(prm), _ptr(theta), _ptr(u),
                             _ptr(x_out), _ptr(resid), int(resid_every), _ptr(wbuf), wbuf.numel(),
                             _stream(dev))
        _check("sci_admm_tv", st)
        return x_out, theta, u, resid
    name = "sci_twist_tv" if twist else ("sci_fista_tv" if fista else "sci_gap_tv")
    st = getattr(lib, name)(_ptr(y), _ptr(bits), nx, ny, B, C.byref(prm), _ptr(theta), _ptr(x_out),
                            _ptr(resid), int(resid_every), _ptr(wbuf), wbuf.numel(), _stream(dev))
    _check(name, st)
    return x_out, theta, resid


def sci_gap_tv(y, bits, B, tv, lam, outer, inner, **kw):
    """GAP-TV (Algorithm 1).  Returns (x^(T), theta^(T), resid-or-None).

    Keyword arguments: storage ('f32'|'bf16'|'f16'); theta (state buffer,
    updated in place: resumed from unless init=True; default a new buffer
    started at Phi^T y); init; x_out; resid; resid_every; fuse_k (an int, or
    'tuned' for the autotuner's cached choice); use_graph;
    work (a Workspace reused across calls); dual ('fgp' or 'cham', the
    TVdenoise box of Algorithm 1); warm_start (carry the box's dual w from
    one TVdenoise call to the next; resuming with init=False continues from
    the w the previous call left in the same work); check_input (count
    NaN / Inf in y, and theta / u when resuming, on the device first and
    raise SciError with SCI_ERR_NONFINITE; the call then waits for the GPU).  Reusing the same
    buffers lets the library replay its cached CUDA graph.
    """
    return _solve(False, y, bits, B, tv, lam, outer, inner, **kw)


def sci_fista_tv(y, bits, B, tv, lam, outer, inner, **kw):
    """FISTA-TV (Sec. 2.2; L = max R, same lambda as GAP).  Returns (x^(T), x^(T), resid-or-None);
    keyword arguments as sci_gap_tv."""
    return _solve(False, y, bits, B, tv, lam, outer, inner, fista=True, **kw)


def sci_twist_tv(y, bits, B, tv, lam, outer, inner, **kw):
    """TwIST-TV (Sec. 2.2; steps on Phi / sqrt(L), alpha and beta from the
    eigenvalue bounds of the normalised Phi^T Phi).  Returns (x^(T), x^(T),
    resid-or-None); keyword arguments as sci_gap_tv."""
    return _solve(False, y, bits, B, tv, lam, outer, inner, twist=True, **kw)


def sci_admm_tv(y, bits, B, tv, lam, rho, outer, inner, **kw):
    """ADMM-TV (Eqs. 24-26).  Returns (x^(T), theta^(T), u^(T), resid-or-None)."""
    return _solve(True, y, bits, B, tv, lam, outer, inner, rho=rho, **kw)


class Batch:
    """Descriptors for sci_gap_tv_batched, kept alive with their buffers.

    ys: list of float32 [nx][ny] measurements; bits: list of packed masks;
    Bs: frame counts.  theta / x_out buffers are allocated once here, so
    repeated solves reuse them (and the library's cached CUDA graph).
    """

    def __init__(self, ys, bits, Bs, x_out=True):
        if not (len(ys) == len(bits) == len(Bs)) or not ys:
            raise ValueError("ys, bits and Bs must be non-empty lists of the same length")
        _need_cuda(*ys, *bits)
        self.ys, self.bits, self.Bs = list(ys), list(bits), [int(b) for b in Bs]
        dev = ys[0].device
        self.thetas = [torch.empty((b, *y.shape), dtype=torch.float32, device=dev) for y, b in zip(ys, Bs)]
        self.x_outs = ([torch.empty_like(t) for t in self.thetas] if x_out else [None] * len(ys))
        arr = (SciProblem * len(ys))()
        for k, (y, bb, b, th, xo) in enumerate(zip(self.ys, self.bits, self.Bs, self.thetas, self.x_outs)):
            arr[k] = SciProblem(y.shape[0], y.shape[1], b, y.data_ptr(), bb.data_ptr(), th.data_ptr(),
                                None if xo is None else xo.data_ptr())
        self.problems = arr
        self.work = Workspace(dev)
        self.device = dev


def sci_gap_tv_batched(batch: Batch, tv, lam, outer, inner, storage="f32", init=True, fuse_k=0,
                       use_graph=True, dual="fgp"):
    """GAP-TV on every measurement of `batch` (results in batch.x_outs / batch.thetas).
    fuse_k='tuned' takes the depth from the autotuner's cache, timing the batch
    first on a miss (which overwrites its buffers, so it needs init=True)."""
    if fuse_k == "tuned":
        if not init:
            raise ValueError("fuse_k='tuned' times probe solves in the batch's buffers: it needs init=True")
        from . import tune
        fuse_k = tune.tuned_batch_fuse(batch, tv, lam, inner, storage=storage, dual=dual)
    prm = _params(tv, lam, 0.0, outer, inner, storage, fuse_k, init, use_graph, dual)
    lib = load()
    n = len(batch.ys)
    need = lib.sci_gap_tv_batched_workspace(batch.problems, n, C.byref(prm))
    if need == 0:
        raise SciError("sci_gap_tv_batched_workspace", 1)
    wbuf = batch.work.get(need)
    _check("sci_gap_tv_batched", lib.sci_gap_tv_batched(batch.problems, n, C.byref(prm), _ptr(wbuf),
                                                        wbuf.numel(), _stream(batch.device)))
    return batch.x_outs, batch.thetas


ALGO = {"gap": 0, "admm": 1, "fista": 2}


def _host_candidates(candidates):
    cands = [int(k) for k in candidates]
    if not cands:
        raise ValueError("no fuse-depth candidates")
    return cands, (C.c_int * len(cands))(*cands), (C.c_float * len(cands))(), C.c_int(0)


def sci_tune_fuse(algo, y, bits, B, tv, lam, inner, candidates, rho=0.0, storage="f32", dual="fgp",
                  probe_iters=2, reps=3, work=None):
    """Times probe_iters outer iterations of the `algo` solve ('gap', 'admm',
    'fista') at each fuse depth in `candidates` (sci_tune_fuse, CUDA events on
    the current stream).  Returns (best candidate, [median ms per candidate]).
    The probe solves run in buffers of their own."""
    _need_cuda(y, bits)
    nx, ny = y.shape
    dev = y.device
    theta = torch.empty((B, nx, ny), dtype=torch.float32, device=dev)
    u = torch.empty_like(theta) if algo == "admm" else None
    prm = _params(tv, lam, rho, probe_iters, inner, storage, 0, True, False, dual)
    lib = load()
    wbuf = (work or Workspace(dev)).get(lib.sci_solver_workspace(nx, ny, B, C.byref(prm)))
    cands, c_arr, ms, best = _host_candidates(candidates)
    _check("sci_tune_fuse", lib.sci_tune_fuse(ALGO[algo], _ptr(y), _ptr(bits), nx, ny, int(B), C.byref(prm),
                                              _ptr(theta), _ptr(u), _ptr(wbuf), wbuf.numel(), c_arr, len(cands),
                                              int(probe_iters), int(reps), ms, C.byref(best), _stream(dev)))
    return int(best.value), [float(v) for v in ms]


def sci_tile_classes(tv: str, B: int) -> list[int]:
    """Tile classes (sci_params.tile) that can run this TV form and frame
    count, the library's default first ([] when none: VTV with B > 24)."""
    out = (C.c_int * 8)()
    n = int(load().sci_tile_classes(TV[tv], int(B), out, 8))
    return [int(out[i]) for i in range(min(n, 8))]


def sci_fused_updates_tile(tv: str, B: int, inner_iters: int, fuse_k: int = 0, tile: int = 0) -> int:
    """Dual updates per fused launch for a tile class (-1: the class does not fit)."""
    return int(load().sci_fused_updates_tile(TV[tv], int(B), int(inner_iters), int(fuse_k), int(tile)))


def sci_tune_launch(algo, y, bits, B, tv, lam, inner, pairs, rho=0.0, storage="f32", dual="fgp",
                    probe_iters=2, reps=3, work=None):
    """sci_tune_fuse over (fuse_k, tile) pairs.  Returns (index of the fastest
    pair, [median ms per pair])."""
    _need_cuda(y, bits)
    nx, ny = y.shape
    dev = y.device
    theta = torch.empty((B, nx, ny), dtype=torch.float32, device=dev)
    u = torch.empty_like(theta) if algo == "admm" else None
    prm = _params(tv, lam, rho, probe_iters, inner, storage, 0, True, False, dual)
    lib = load()
    wbuf = (work or Workspace(dev)).get(lib.sci_solver_workspace(nx, ny, B, C.byref(prm)))
    n = len(pairs)
    ks = (C.c_int * n)(*[int(k) for k, _ in pairs])
    ts = (C.c_int * n)(*[int(t) for _, t in pairs])
    ms = (C.c_float * n)()
    best = C.c_int(0)
    _check("sci_tune_launch", lib.sci_tune_launch(ALGO[algo], _ptr(y), _ptr(bits), nx, ny, int(B), C.byref(prm),
                                                  _ptr(theta), _ptr(u), _ptr(wbuf), wbuf.numel(), ks, ts, n,
                                                  int(probe_iters), int(reps), ms, C.byref(best), _stream(dev)))
    return int(best.value), [float(v) for v in ms]


def sci_tune_fuse_batched(batch: Batch, tv, lam, inner, candidates, storage="f32", dual="fgp",
                          probe_iters=1, reps=3):
    """sci_tune_fuse for sci_gap_tv_batched on `batch` (one depth for the whole
    batch; overwrites batch.thetas and batch.x_outs).  Returns (best, [ms])."""
    prm = _params(tv, lam, 0.0, probe_iters, inner, storage, 0, True, False, dual)
    lib = load()
    n = len(batch.ys)
    need = lib.sci_gap_tv_batched_workspace(batch.problems, n, C.byref(prm))
    if need == 0:
        raise SciError("sci_gap_tv_batched_workspace", 1)
    wbuf = batch.work.get(need)
    cands, c_arr, ms, best = _host_candidates(candidates)
    _check("sci_tune_fuse_batched",
           lib.sci_tune_fuse_batched(batch.problems, n, C.byref(prm), _ptr(wbuf), wbuf.numel(), c_arr, len(cands),
                                     int(probe_iters), int(reps), ms, C.byref(best), _stream(batch.device)))
    return int(best.value), [float(v) for v in ms]


def sci_conv3d_c32_bf16(act: torch.Tensor, w: torch.Tensor, bias: torch.Tensor | None = None,
                        relu: bool = False):
    """3x3x3 conv, 32 -> 32 channels, on the tensor cores: act BF16 [n][D][H][W][32],
    w BF16 [27][32][32] -> BF16 [n][D][H][W][32] (and the kernel's error word)."""
    _need_cuda(act, w, bias)
    if act.dtype != torch.bfloat16 or w.dtype != torch.bfloat16 or act.shape[-1] != 32:
        raise ValueError("act and w must be bfloat16 with 32 channels")
    n, D, H, W, _ = act.shape
    out = torch.empty_like(act)
    err = torch.zeros(1, dtype=torch.int32, device=act.device)
    _check("sci_conv3d_c32_bf16", load().sci_conv3d_c32_bf16(_ptr(act), _ptr(w), _ptr(bias), int(relu), n, D,
                                                             H, W, _ptr(out), _ptr(err), _stream(act.device)))
    return out, err


class LearnedProx:
    """FP32 master parameters, Adam state and scratch of the learned prox."""

    def __init__(self, device="cuda", params: torch.Tensor | None = None):
        self.device = torch.device(device)
        n = int(load().sci_lprox_param_count())
        self.params = (params.clone() if params is not None
                       else torch.zeros(n, dtype=torch.float32, device=self.device))
        if self.params.numel() != n:
            raise ValueError(f"expected {n} parameters")
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0
        self.work = Workspace(self.device)

    @staticmethod
    def param_count() -> int:
        return int(load().sci_lprox_param_count())

    def apply(self, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """theta = x + f(x) for x float32 [count][B][nx][ny] (or [B][nx][ny])."""
        _need_cuda(x)
        xv = x if x.dim() == 4 else x.unsqueeze(0)
        count, B, nx, ny = xv.shape
        lib = load()
        wbuf = self.work.get(lib.sci_lprox_workspace(nx, ny, B, count, 0))
        theta = torch.empty_like(x) if out is None else out
        _check("sci_lprox_apply", lib.sci_lprox_apply(_ptr(self.params), _ptr(x), nx, ny, B, count, _ptr(theta),
                                                      _ptr(wbuf), wbuf.numel(), _stream(x.device)))
        return theta

    def train_step(self, x: torch.Tensor, target: torch.Tensor, lr: float) -> torch.Tensor:
        """One Adam step; returns the pre-step sum of squared errors (device double)."""
        _need_cuda(x, target)
        count, B, nx, ny = x.shape
        lib = load()
        wbuf = self.work.get(lib.sci_lprox_workspace(nx, ny, B, count, 1))
        loss = torch.zeros(1, dtype=torch.float64, device=x.device)
        self.step += 1
        _check("sci_lprox_train_step", lib.sci_lprox_train_step(
            _ptr(self.params), _ptr(self.m), _ptr(self.v), self.step, float(lr), _ptr(x), _ptr(target), nx, ny,
            B, count, _ptr(loss), _ptr(wbuf), wbuf.numel(), _stream(x.device)))
        return loss

    def grads(self, x: torch.Tensor, target: torch.Tensor):
        _need_cuda(x, target)
        count, B, nx, ny = x.shape
        lib = load()
        wbuf = self.work.get(lib.sci_lprox_workspace(nx, ny, B, count, 1))
        g = torch.empty_like(self.params)
        loss = torch.zeros(1, dtype=torch.float64, device=x.device)
        _check("sci_lprox_grads", lib.sci_lprox_grads(_ptr(self.params), _ptr(x), _ptr(target), nx, ny, B, count,
                                                      _ptr(g), _ptr(loss), _ptr(wbuf), wbuf.numel(),
                                                      _stream(x.device)))
        return g, loss

    def error_word(self, x_shape, training: bool) -> int:
        count, B, nx, ny = x_shape
        lib = load()
        wbuf = self.work.get(lib.sci_lprox_workspace(nx, ny, B, count, int(training)))
        ptr = C.c_void_p()
        _check("sci_lprox_error_word", lib.sci_lprox_error_word(_ptr(wbuf), wbuf.numel(), nx, ny, B, count,
                                                                int(training), C.byref(ptr)))
        off = int(ptr.value) - wbuf.data_ptr()
        return int(wbuf[off:off + 4].view(torch.int32).item())


def sci_gap_tv_lprox(net: "LearnedProx", y: torch.Tensor, bits: torch.Tensor, B: int, outer: int,
                     plain_tv: str = "vtv", plain_lam: float = 0.05, plain_inner: int = 10,
                     check_every: int = 0, resid_limit=None, ratio: float = 1.05, theta=None, x_out=None,
                     work: Workspace | None = None):
    """GAP-TV with the learned prox on y [count][nx][ny] (bits likewise).

    Returns (x^(T), theta^(T), fell_back list, residual history [count][checks]).
    With check_every > 0 and resid_limit (the plain method's residual at each
    checkpoint), measurements whose residual exceeds ratio x limit restart
    from their last checkpoint with plain GAP-TV (plain_tv, plain_lam,
    plain_inner FGP updates).
    """
    _need_cuda(y, bits, theta, x_out)
    count, nx, ny = y.shape
    dev = y.device
    init = theta is None
    if theta is None:
        theta = torch.empty((count, B, nx, ny), dtype=torch.float32, device=dev)
    if x_out is None:
        x_out = torch.empty_like(theta)
    plain = _params(plain_tv, plain_lam, 0.0, outer, plain_inner, "f32", 0, 0, 0)
    lib = load()
    need = lib.sci_gap_tv_lprox_workspace(nx, ny, B, count, C.byref(plain))
    wbuf = (work or Workspace(dev)).get(need)
    nchk = (outer + check_every - 1) // check_every if check_every > 0 else 0
    lim = None
    if resid_limit is not None:
        lim = (C.c_double * len(resid_limit))(*[float(v) for v in resid_limit])
    fell = (C.c_int * count)()
    rout = (C.c_double * max(1, count * nchk))()
    _check("sci_gap_tv_lprox", lib.sci_gap_tv_lprox(
        _ptr(net.params), _ptr(y), _ptr(bits), nx, ny, B, count, int(outer), int(init), _ptr(theta), _ptr(x_out),
        int(check_every), lim, float(ratio), C.byref(plain), fell, rout, _ptr(wbuf), wbuf.numel(), _stream(dev)))
    hist = [[rout[v * nchk + c] for c in range(nchk)] for v in range(count)]
    return x_out, theta, [int(f) for f in fell], hist


def sci_last_batch_launches() -> int:
    return int(load().sci_last_batch_launches())


def sci_graph_cache_clear():
    load().sci_graph_cache_clear()


def sci_fused_updates(tv: str, B: int, inner_iters: int, fuse_k: int = 0) -> int:
    """Dual updates per fused launch the library uses (0: per-update kernels)."""
    return int(load().sci_fused_updates(TV[tv], int(B), int(inner_iters), int(fuse_k)))


def sci_last_solve_launches() -> int:
    """Kernels enqueued by this thread's most recent solve call."""
    return int(load().sci_last_solve_launches())


def sci_sqdiff_f64(a: torch.Tensor, b: torch.Tensor | None = None,
                   work: Workspace | None = None) -> torch.Tensor:
    """sum (a - b)^2 (or sum a^2) with FP64 accumulation; a 1-element device double tensor."""
    _need_cuda(a, b)
    lib = load()
    out = torch.empty(1, dtype=torch.float64, device=a.device)
    wbuf = (work or Workspace(a.device)).get(lib.sci_reduce_workspace())
    _check("sci_sqdiff_f64", lib.sci_sqdiff_f64(_ptr(a), _ptr(b), a.numel(), _ptr(out), _ptr(wbuf),
                                                wbuf.numel(), _stream(a.device)))
    return out


def sci_residual_f64(theta: torch.Tensor, y: torch.Tensor, bits: torch.Tensor,
                     work: Workspace | None = None) -> torch.Tensor:
    """||y - Phi theta||^2 with FP64 accumulation; a 1-element device double tensor."""
    _need_cuda(theta, y, bits)
    B, nx, ny = theta.shape
    lib = load()
    out = torch.empty(1, dtype=torch.float64, device=theta.device)
    wbuf = (work or Workspace(theta.device)).get(lib.sci_reduce_workspace())
    _check("sci_residual_f64", lib.sci_residual_f64(_ptr(theta), _ptr(y), _ptr(bits), nx, ny, B, _ptr(out),
                                                    _ptr(wbuf), wbuf.numel(), _stream(theta.device)))
    return out
