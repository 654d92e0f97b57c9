"""Launch-shape autotuner driver (fuse depth and tile class) with a JSON cache.

How many FGP dual updates K one temporally blocked launch runs decides the
tile's halo, hence the useful share of every tile, against the number of
launches per TVdenoise (ceil(S / K)).  The best K depends on the frame size,
the frame count (which fixes the tile class), S, the storage type and the GPU.
The library's sci_tune_fuse / sci_tune_fuse_batched time short solves at each
candidate with CUDA events on the launching stream; this module picks the
candidates (the distinct depths the library would actually run), keys the
winner by everything that decides it and keeps it in a JSON file, so later
runs on the same GPU model reuse it without timing.  With FP32 storage
every K gives bit-identical results, so the cache changes speed, never
output; with 16-bit storage the duals carried from one launch to the next are
rounded to 16 bits, and K moves those roundings.

The tile class (sci_params.tile) is tuned beside K for single solves
(tuned_launch): each class that fits the TV form and frame count trades the
tile's area, hence its useful share at a given halo, against the threads and
registers one CTA holds.

The cache file is $SCI_TUNE_CACHE, else ~/.cache/paper_2005_08028_gb300/fuse.json.
"""
from __future__ import annotations

import collections
import hashlib
import json
import os
import tempfile
import threading

import torch

from . import sci as S

_lock = threading.Lock()


def default_cache_path() -> str:
    return os.environ.get("SCI_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "paper_2005_08028_gb300", "fuse.json")


class FuseCache:
    """Tuned depths by key, persisted as one JSON object {key: entry}."""

    def __init__(self, path: str | None = None):
        self.path = path or default_cache_path()
        self._d = self._load()

    def _load(self) -> dict:
        try:
            with open(self.path) as f:
                d = json.load(f)
            return d if isinstance(d, dict) else {}
        except (OSError, ValueError):
            return {}

    def get(self, key: str) -> int | None:
        e = self._d.get(key)
        if isinstance(e, dict) and isinstance(e.get("fuse_k"), int):
            return e["fuse_k"]
        return None

    def get_launch(self, key: str) -> tuple[int, int] | None:
        e = self._d.get(key)
        if isinstance(e, dict) and isinstance(e.get("fuse_k"), int) and isinstance(e.get("tile"), int):
            return e["fuse_k"], e["tile"]
        return None

    def put_launch(self, key: str, pair: tuple[int, int], candidates: list[tuple[int, int]],
                   ms: list[float]) -> None:
        """Store one (fuse_k, tile) entry, merging as put does."""
        merged = self._load()
        merged.update(self._d)
        merged[key] = {"fuse_k": int(pair[0]), "tile": int(pair[1]),
                       "candidates": [[int(k), int(t)] for k, t in candidates],
                       "ms": [round(float(m), 6) for m in ms]}
        self._d = merged
        self.save()

    def put(self, key: str, fuse_k: int, candidates: list[int], ms: list[float]) -> None:
        """Store one entry.  The file is read again first, so entries that
        another process stored since this cache was loaded are kept."""
        merged = self._load()
        merged.update(self._d)
        merged[key] = {"fuse_k": int(fuse_k), "candidates": [int(c) for c in candidates],
                       "ms": [round(float(m), 6) for m in ms]}
        self._d = merged
        self.save()

    def save(self) -> None:
        d = os.path.dirname(os.path.abspath(self.path))
        os.makedirs(d, exist_ok=True)
        fd, tmp = tempfile.mkstemp(dir=d, prefix=".fuse-", suffix=".json")
        with os.fdopen(fd, "w") as f:
            json.dump(self._d, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)  # readers see the old or the new file, never half of one

    def __len__(self) -> int:
        return len(self._d)


def device_name(dev: torch.device) -> str:
    return torch.cuda.get_device_name(dev) if dev.type == "cuda" else dev.type


def solve_key(gpu: str, algo: str, tv: str, nx: int, ny: int, B: int, inner: int, storage: str,
              dual: str) -> str:
    return f"{gpu}|{algo}|{tv}|{nx}x{ny}x{B}|S{inner}|{storage}|{dual}"


def batch_key(gpu: str, tv: str, sizes: list[tuple[int, int, int]], inner: int, storage: str, dual: str) -> str:
    """Key of a batch: the multiset of its (nx, ny, B), order-free."""
    mix = ",".join(f"{nx}x{ny}x{b}*{c}" for (nx, ny, b), c in sorted(collections.Counter(sizes).items()))
    if len(mix) > 160:
        mix = "sha1:" + hashlib.sha1(mix.encode()).hexdigest()
    return f"{gpu}|batched|{tv}|{mix}|S{inner}|{storage}|{dual}"


def fuse_candidates(tv: str, B: int, inner: int, per_update: bool = True) -> list[int]:
    """The distinct depths the library runs for this TV, frame count and S:
    its default first (so a tie keeps it), then deepest to shallowest, then
    -1 (one launch per update) when per_update."""
    out = []
    for k in [0] + list(range(inner, 0, -1)):
        eff = S.sci_fused_updates(tv, B, inner, k)
        if eff > 0 and eff not in out:
            out.append(eff)
    if per_update:
        out.append(-1)
    return out


def launch_candidates(tv: str, B: int, inner: int, per_update: bool = True) -> list[tuple[int, int]]:
    """(fuse_k, tile) pairs giving the distinct launch shapes the library can
    run for this TV form, frame count and S: the library's default (0, 0)
    first, then every tile class that fits with each distinct depth (deepest
    first), then (-1, 0) (one launch per update) when per_update."""
    classes = S.sci_tile_classes(tv, int(B))
    default = (S.sci_fused_updates(tv, int(B), int(inner), 0), classes[0] if classes else 0)
    out, seen = [(0, 0)], {default}
    for c in classes:
        for k in range(int(inner), 0, -1):
            eff = S.sci_fused_updates_tile(tv, int(B), int(inner), k, c)
            if eff > 0 and (eff, c) not in seen:
                seen.add((eff, c))
                out.append((eff, c))
    if per_update:
        out.append((-1, 0))
    return out


def tuned_launch(algo: str, y: torch.Tensor, bits: torch.Tensor, B: int, tv: str, lam: float, inner: int, *,
                 rho: float = 0.0, storage: str = "f32", dual: str = "fgp", cache: FuseCache | None = None,
                 probe_iters: int = 2, reps: int = 3, timer=None, work=None) -> tuple[int, int]:
    """(fuse_k, tile) for this solve: the cached choice, else timed over
    launch_candidates (timer defaults to sci.sci_tune_launch) and stored."""
    nx, ny = int(y.shape[0]), int(y.shape[1])
    with _lock:
        cache = cache if cache is not None else FuseCache()
        key = solve_key(device_name(y.device), algo, tv, nx, ny, int(B), int(inner), storage, dual) + "|launch"
        got = cache.get_launch(key)
        if got is not None:
            return got
        cands = launch_candidates(tv, int(B), int(inner))
        if len(cands) == 1:
            best, ms = 0, [0.0]
        else:
            kw = {} if work is None else {"work": work}
            best, ms = (timer or S.sci_tune_launch)(algo, y, bits, B, tv, lam, inner, cands, rho=rho,
                                                    storage=storage, dual=dual, probe_iters=probe_iters,
                                                    reps=reps, **kw)
        cache.put_launch(key, cands[best], cands, ms)
        return cands[best]


def batch_fuse_candidates(tv: str, Bs: list[int], inner: int) -> list[int]:
    """fuse_k values for a batch that give distinct per-class depths: 0 (the
    library default) first, then deepest to shallowest."""
    classes = sorted(set(int(b) for b in Bs))
    out, seen = [], set()
    for k in [0] + list(range(inner, 0, -1)):
        depths = tuple(S.sci_fused_updates(tv, b, inner, k) for b in classes)
        if depths not in seen:
            seen.add(depths)
            out.append(k)
    return out


def tuned_fuse(algo: str, y: torch.Tensor, bits: torch.Tensor, B: int, tv: str, lam: float, inner: int, *,
               rho: float = 0.0, storage: str = "f32", dual: str = "fgp", cache: FuseCache | None = None,
               probe_iters: int = 2, reps: int = 3, timer=None, work=None) -> int:
    """fuse_k for this solve: the cached choice, else timed (timer defaults to
    sci.sci_tune_fuse, with the same arguments; ``work``, a sci.Workspace,
    is lent to the probe solves) and stored."""
    nx, ny = int(y.shape[0]), int(y.shape[1])
    with _lock:
        cache = cache if cache is not None else FuseCache()
        key = solve_key(device_name(y.device), algo, tv, nx, ny, int(B), int(inner), storage, dual)
        k = cache.get(key)
        if k is not None:
            return k
        cands = fuse_candidates(tv, int(B), int(inner))
        if len(cands) == 1:
            best, ms = cands[0], [0.0]
        else:
            kw = {} if work is None else {"work": work}
            best, ms = (timer or S.sci_tune_fuse)(algo, y, bits, B, tv, lam, inner, cands, rho=rho,
                                                  storage=storage, dual=dual, probe_iters=probe_iters, reps=reps,
                                                  **kw)
        cache.put(key, best, cands, ms)
        return best


def tuned_batch_fuse(batch, tv: str, lam: float, inner: int, *, storage: str = "f32", dual: str = "fgp",
                     cache: FuseCache | None = None, probe_iters: int = 1, reps: int = 3, timer=None) -> int:
    """fuse_k for sci_gap_tv_batched on this batch: cached, else timed in the
    batch's own buffers (overwriting them) and stored."""
    sizes = [(int(y.shape[0]), int(y.shape[1]), int(b)) for y, b in zip(batch.ys, batch.Bs)]
    with _lock:
        cache = cache if cache is not None else FuseCache()
        key = batch_key(device_name(batch.device), tv, sizes, int(inner), storage, dual)
        k = cache.get(key)
        if k is not None:
            return k
        cands = batch_fuse_candidates(tv, batch.Bs, int(inner))
        if len(cands) == 1:
            best, ms = cands[0], [0.0]
        else:
            best, ms = (timer or S.sci_tune_fuse_batched)(batch, tv, lam, inner, cands, storage=storage,
                                                          dual=dual, probe_iters=probe_iters, reps=reps)
        cache.put(key, best, cands, ms)
        return best
