"""CPU checks of the fuse-depth autotuner: candidate choice, cache keys, the
JSON cache file, the cache-hit path (no timing), and the C ABI's argument
checks, which return before any CUDA call.  Timing itself is covered by
tests/test_gpu_tune.py."""
import ctypes as C
import json
import os
import types

import pytest
import torch

from paper_2005_08028_gb300 import sci as S
from paper_2005_08028_gb300 import tune

ARG = 1  # SCI_ERR_ARG


@pytest.fixture(scope="module")
def lib():
    from paper_2005_08028_gb300 import build as b
    return S.load(b.build())


class FakeTimer:
    """Stands in for sci_tune_fuse(_batched): records calls, prefers one depth."""

    def __init__(self, prefer):
        self.prefer, self.calls = prefer, []

    def __call__(self, *args, **kw):
        cands = args[7] if len(args) > 7 else args[4]
        self.calls.append((list(cands), kw))
        ms = [1.0 if c == self.prefer else 2.0 + i for i, c in enumerate(cands)]
        return (self.prefer if self.prefer in cands else cands[0]), ms


@pytest.mark.parametrize("tv", ["atv", "itv2d", "vtv"])
@pytest.mark.parametrize("B", [1, 8, 10, 16, 24])
@pytest.mark.parametrize("inner", [1, 5, 10])
def test_candidates_are_the_distinct_depths_the_library_runs(lib, tv, B, inner):
    c = tune.fuse_candidates(tv, B, inner)
    assert c[0] == S.sci_fused_updates(tv, B, inner, 0)  # the default first: a tie keeps it
    assert c[-1] == -1 and len(set(c)) == len(c)
    for k in c[:-1]:
        assert 1 <= k <= inner and S.sci_fused_updates(tv, B, inner, k) == k
    # every depth the library can run for fuse_k = 1..inner is offered
    assert {S.sci_fused_updates(tv, B, inner, k) for k in range(1, inner + 1)} == set(c[:-1])


def test_no_fused_kernel_leaves_the_per_update_path_only(lib):
    assert tune.fuse_candidates("vtv", 32, 10) == [-1]
    assert tune.fuse_candidates("vtv", 32, 10, per_update=False) == []


def test_batch_candidates_give_distinct_per_class_depths(lib):
    Bs = [8, 8, 10, 24]
    c = tune.batch_fuse_candidates("vtv", Bs, 10)
    assert c[0] == 0
    depths = [tuple(S.sci_fused_updates("vtv", b, 10, k) for b in sorted(set(Bs))) for k in c]
    assert len(set(depths)) == len(depths)
    every = {tuple(S.sci_fused_updates("vtv", b, 10, k) for b in sorted(set(Bs))) for k in range(0, 11)}
    assert set(depths) == every


def test_batch_key_ignores_order_and_hashes_long_mixes():
    a = tune.batch_key("g", "vtv", [(64, 64, 8), (128, 96, 10), (64, 64, 8)], 5, "f16", "fgp")
    b = tune.batch_key("g", "vtv", [(128, 96, 10), (64, 64, 8), (64, 64, 8)], 5, "f16", "fgp")
    assert a == b and "64x64x8*2" in a
    assert a != tune.batch_key("g", "vtv", [(64, 64, 8), (128, 96, 10)], 5, "f16", "fgp")
    long = tune.batch_key("g", "vtv", [(n, n, 8) for n in range(16, 80)], 5, "f16", "fgp")
    assert "sha1:" in long and len(long) < 120


def test_cache_round_trip_and_atomic_file(tmp_path):
    p = str(tmp_path / "sub" / "fuse.json")
    c = tune.FuseCache(p)
    assert len(c) == 0 and c.get("k") is None
    c.put("k", 5, [6, 5, -1], [0.2, 0.1, 0.9])
    assert tune.FuseCache(p).get("k") == 5
    assert json.load(open(p))["k"]["candidates"] == [6, 5, -1]
    assert sorted(os.listdir(tmp_path / "sub")) == ["fuse.json"]  # no temporary file left


def test_two_writers_keep_each_others_entries(tmp_path):
    p = str(tmp_path / "fuse.json")
    a, b = tune.FuseCache(p), tune.FuseCache(p)  # both loaded before either wrote
    a.put("ka", 4, [4, -1], [0.1, 0.2])
    b.put("kb", 6, [6, -1], [0.3, 0.4])
    a.put("kc", 2, [2, -1], [0.5, 0.6])
    c = tune.FuseCache(p)
    assert (c.get("ka"), c.get("kb"), c.get("kc")) == (4, 6, 2)


def test_unreadable_or_foreign_cache_starts_empty(tmp_path):
    p = tmp_path / "fuse.json"
    p.write_text("{not json")
    assert len(tune.FuseCache(str(p))) == 0
    p.write_text("[1, 2]")
    assert len(tune.FuseCache(str(p))) == 0
    p.write_text(json.dumps({"k": {"fuse_k": "five"}}))
    assert tune.FuseCache(str(p)).get("k") is None


def test_env_var_names_the_cache(monkeypatch, tmp_path):
    monkeypatch.setenv("SCI_TUNE_CACHE", str(tmp_path / "x.json"))
    assert tune.default_cache_path() == str(tmp_path / "x.json")


def test_tuned_fuse_times_once_then_hits_the_cache(lib, tmp_path):
    cache = tune.FuseCache(str(tmp_path / "f.json"))
    y, bits = torch.zeros(40, 56), torch.zeros(40, 56, dtype=torch.int32)
    t = FakeTimer(prefer=5)
    k = tune.tuned_fuse("gap", y, bits, 8, "vtv", 0.05, 10, cache=cache, timer=t)
    assert k == 5 and len(t.calls) == 1
    assert t.calls[0][0] == tune.fuse_candidates("vtv", 8, 10)
    assert tune.tuned_fuse("gap", y, bits, 8, "vtv", 0.05, 10, cache=cache, timer=t) == 5
    assert len(t.calls) == 1  # cache hit: nothing timed
    # a fresh cache object reads the stored choice from the file
    assert tune.tuned_fuse("gap", y, bits, 8, "vtv", 0.05, 10, cache=tune.FuseCache(cache.path), timer=t) == 5
    assert len(t.calls) == 1
    # what decides the depth is in the key: another storage type is timed again
    tune.tuned_fuse("gap", y, bits, 8, "vtv", 0.05, 10, storage="f16", cache=cache, timer=t)
    tune.tuned_fuse("admm", y, bits, 8, "vtv", 0.05, 10, rho=0.01, cache=cache, timer=t)
    tune.tuned_fuse("gap", y, bits, 8, "vtv", 0.05, 5, cache=cache, timer=t)
    assert len(t.calls) == 4 and t.calls[2][1]["rho"] == 0.01


def test_the_callers_workspace_is_lent_to_the_probes(lib, tmp_path):
    cache = tune.FuseCache(str(tmp_path / "f.json"))
    t = FakeTimer(prefer=6)
    y = torch.zeros(16, 16)
    ws = object()
    tune.tuned_fuse("gap", y, y, 8, "vtv", 0.05, 10, cache=cache, timer=t, work=ws)
    assert t.calls[0][1]["work"] is ws
    tune.tuned_fuse("gap", y, y, 8, "vtv", 0.05, 5, cache=cache, timer=t)
    assert "work" not in t.calls[1][1]


def test_a_single_candidate_is_not_timed(lib, tmp_path):
    cache = tune.FuseCache(str(tmp_path / "f.json"))
    t = FakeTimer(prefer=3)
    y = torch.zeros(16, 16)
    assert tune.tuned_fuse("gap", y, y, 32, "vtv", 0.05, 10, cache=cache, timer=t) == -1
    assert t.calls == []


def test_tuned_batch_fuse_keys_the_size_mix(lib, tmp_path):
    cache = tune.FuseCache(str(tmp_path / "f.json"))
    batch = types.SimpleNamespace(ys=[torch.zeros(64, 64), torch.zeros(96, 80)], Bs=[8, 24],
                                  device=torch.device("cpu"))
    t = FakeTimer(prefer=4)
    assert tune.tuned_batch_fuse(batch, "vtv", 0.05, 10, cache=cache, timer=t) == 4
    assert t.calls[0][0] == tune.batch_fuse_candidates("vtv", [8, 24], 10)
    batch.ys.reverse(); batch.Bs.reverse()
    assert tune.tuned_batch_fuse(batch, "vtv", 0.05, 10, cache=cache, timer=t) == 4
    assert len(t.calls) == 1


def test_c_abi_rejects_bad_tuner_arguments_before_any_launch(lib):
    fake = C.c_void_p(0x10000)  # never dereferenced: validation fails first
    prm = S.SciParams(0, 0.05, 0.0, 10, 5, 0, 0, 1, 1, 0)
    cands = (C.c_int * 3)(5, 2, -1)
    ms = (C.c_float * 3)()
    best = C.c_int(0)

    def tune_call(algo=0, params=C.byref(prm), c=cands, n=3, probe=2, reps=3, msp=ms, bestp=C.byref(best), u=None):
        return lib.sci_tune_fuse(algo, fake, fake, 8, 8, 2, params, fake, u, fake, 1 << 30, c, n, probe, reps,
                                 msp, bestp, None)

    assert tune_call(params=None) == ARG
    assert tune_call(n=0) == ARG and tune_call(n=65) == ARG
    assert tune_call(c=(C.c_int * 3)(5, -2, 1)) == ARG
    assert tune_call(c=None) == ARG and tune_call(msp=None) == ARG and tune_call(bestp=None) == ARG
    assert tune_call(reps=0) == ARG and tune_call(reps=101) == ARG
    assert tune_call(probe=0) == ARG and tune_call(probe=1001) == ARG
    assert tune_call(algo=3) == ARG and tune_call(algo=-1) == ARG
    assert tune_call(algo=1) == ARG  # ADMM without u
    probs = (S.SciProblem * 1)()
    assert lib.sci_tune_fuse_batched(probs, 1, None, fake, 1 << 30, cands, 3, 1, 3, ms, C.byref(best), None) == ARG
    assert lib.sci_tune_fuse_batched(probs, 1, C.byref(prm), fake, 1 << 30, cands, 0, 1, 3, ms, C.byref(best),
                                     None) == ARG
    assert best.value == 0  # untouched on error


def test_bench_tuning_section_reports_choices_and_failures(lib):
    import bench
    c = {"B": 10, "inner": 10, "lam": 0.05, "rho": 0.01}
    calls = []

    class Fake:
        sci_fused_updates = staticmethod(S.sci_fused_updates)

        @staticmethod
        def sci_tune_launch(algo, y, bits, B, tv, lam, inner, cands, rho=0.0, probe_iters=2, reps=3):
            calls.append((algo, tv, rho, probe_iters, reps))
            return 0, [1.0 + i for i in range(len(cands))]

    out = bench._fuse_tuning(Fake, c, None, None)
    assert set(out) == {"probe"} | {f"{a}_{t}" for a, t in bench.COMBOS}
    assert out["gap_vtv"]["best"] == out["gap_vtv"]["default"] == [0, 0]
    assert out["gap_vtv"]["default_depth"] == S.sci_fused_updates("vtv", 10, 10, 0)
    assert list(out["admm_atv"]["ms"]) == [f"{k}@{t}" for k, t in tune.launch_candidates("atv", 10, 10)]
    assert [r for _, _, r, _, _ in calls] == [0.0] * 3 + [0.01] * 3

    class Broken:
        sci_fused_updates = staticmethod(S.sci_fused_updates)

        @staticmethod
        def sci_tune_launch(*a, **k):
            raise S.SciError("sci_tune_launch", 3)

    assert "SCI_ERR_CUDA" in bench._fuse_tuning(Broken, c, None, None)["error"]


@pytest.mark.parametrize("tv", ["atv", "itv2d", "vtv"])
@pytest.mark.parametrize("B", [1, 8, 10, 16, 24])
@pytest.mark.parametrize("inner", [1, 5, 10])
def test_launch_candidates_cover_every_class_and_depth(lib, tv, B, inner):
    c = tune.launch_candidates(tv, B, inner)
    assert c[0] == (0, 0) and c[-1] == (-1, 0) and len(set(c)) == len(c)
    classes = S.sci_tile_classes(tv, B)
    assert classes[0] == (1 if tv != "vtv" else min(x for x in (8, 10, 16, 24) if x >= B))
    for k, t in c[1:-1]:
        assert t in classes and 1 <= k <= inner and S.sci_fused_updates_tile(tv, B, inner, k, t) == k
    for t in classes:  # every class is offered (unless its only depth is the default's)
        depths = {S.sci_fused_updates_tile(tv, B, inner, k, t) for k in range(1, inner + 1)}
        offered = {k for k, tt in c if tt == t}
        default = (S.sci_fused_updates(tv, B, inner, 0), classes[0])
        assert depths - offered <= ({default[0]} if t == default[1] else set())


def test_tile_class_queries(lib):
    assert S.sci_tile_classes("atv", 10) == [1, 2, 3, 4] and S.sci_tile_classes("itv2d", 3) == [1, 2, 3, 4]
    assert S.sci_tile_classes("vtv", 8) == [8, 10, 16, 24]
    assert S.sci_tile_classes("vtv", 11) == [16, 24] and S.sci_tile_classes("vtv", 25) == []
    assert S.sci_fused_updates_tile("vtv", 12, 10, 0, 10) == -1  # 12 frames do not fit a 10-frame tile
    assert S.sci_fused_updates_tile("vtv", 8, 10, 10, 16) == 3   # 32 x 16 tiles: halo <= 4
    assert S.sci_fused_updates_tile("atv", 8, 20, 20, 2) == 11   # 32 x 64 tiles: halo <= 12
    assert S.sci_fused_updates_tile("atv", 8, 10, 0, 8) == -1    # a VTV class for ATV


def test_tuned_launch_caches_the_pair(lib, tmp_path):
    cache = tune.FuseCache(str(tmp_path / "f.json"))
    y = torch.zeros(64, 64)
    calls = []

    def timer(algo, yy, bb, B, tv, lam, inner, pairs, **kw):
        calls.append(list(pairs))
        i = pairs.index((3, 2)) if (3, 2) in pairs else 0
        return i, [1.0 if j == i else 2.0 for j in range(len(pairs))]

    assert tune.tuned_launch("gap", y, y, 4, "atv", 0.05, 10, cache=cache, timer=timer) == (3, 2)
    assert tune.tuned_launch("gap", y, y, 4, "atv", 0.05, 10, cache=cache, timer=timer) == (3, 2)
    assert len(calls) == 1 and calls[0] == tune.launch_candidates("atv", 4, 10)
    again = tune.FuseCache(str(tmp_path / "f.json"))
    key = tune.solve_key(tune.device_name(y.device), "gap", "atv", 64, 64, 4, 10, "f32", "fgp") + "|launch"
    assert again.get_launch(key) == (3, 2)


def test_c_abi_rejects_bad_tiles_before_any_launch(lib):
    fake = C.c_void_p(0x10000)
    big = 1 << 40
    for tv, B, tile in ((2, 12, 10), (0, 4, 8), (1, 4, 5), (2, 4, 3), (0, 4, -1)):
        prm = S.SciParams(tv, 0.05, 0.0, 10, 5, 0, 0, 1, 1, 0, 0, 0, tile)
        assert lib.sci_gap_tv(fake, fake, 8, 8, B, C.byref(prm), fake, fake, None, 0, fake, big, None) == 1
    ks = (C.c_int * 2)(0, 3)
    ts = (C.c_int * 2)(0, -1)
    ms = (C.c_float * 2)()
    best = C.c_int(0)
    prm = S.SciParams(0, 0.05, 0.0, 10, 5, 0, 0, 1, 1, 0, 0, 0, 0)
    assert lib.sci_tune_launch(0, fake, fake, 8, 8, 2, C.byref(prm), fake, None, fake, big, ks, ts, 2, 2, 3, ms,
                               C.byref(best), None) == 1
    assert lib.sci_tune_launch(0, fake, fake, 8, 8, 2, C.byref(prm), fake, None, fake, big, ks, None, 2, 2, 3, ms,
                               C.byref(best), None) == 1
