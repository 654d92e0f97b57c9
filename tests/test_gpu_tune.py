"""GPU: the fuse-depth autotuner.  sci_tune_fuse / sci_tune_fuse_batched time
short solves at each candidate depth with CUDA events; a solve with
fuse_k='tuned' takes the winner from the JSON cache (timing on a miss) and,
with FP32 storage, must give bit for bit what the default depth gives, since
every depth does."""
import json

import numpy as np
import pytest

from gpu_helpers import lib, make_problem, to_dev, torch
from paper_2005_08028_gb300 import tune

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    return lib()


@pytest.mark.parametrize("algo", ["gap", "admm", "fista"])
@pytest.mark.parametrize("tv,nx,ny,B", [("atv", 130, 150, 8), ("vtv", 97, 131, 10), ("vtv", 64, 80, 24)])
def test_tuner_times_every_candidate(pkg, algo, tv, nx, ny, B):
    case, y = make_problem(nx, ny, B, 7 + nx, sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    cands = tune.fuse_candidates(tv, B, 10)
    best, ms = pkg.sci_tune_fuse(algo, to_dev(y), bits, B, tv, 0.05, 10, cands,
                                 rho=0.01 if algo == "admm" else 0.0, reps=2)
    assert best in cands and len(ms) == len(cands)
    assert all(np.isfinite(m) and m > 0 for m in ms)
    assert ms[cands.index(best)] == min(ms)


@pytest.mark.parametrize("algo,tv,B", [("gap", "vtv", 8), ("admm", "itv2d", 6), ("fista", "atv", 4)])
def test_tuned_solve_is_bitwise_the_default_solve(pkg, monkeypatch, tmp_path, algo, tv, B):
    path = tmp_path / "fuse.json"
    monkeypatch.setenv("SCI_TUNE_CACHE", str(path))
    case, y = make_problem(200, 330, B, 5 + B, sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    yd = to_dev(y)

    def solve(**kw):
        if algo == "admm":
            return pkg.sci_admm_tv(yd, bits, B, tv, 0.05, 0.01, 6, 10, **kw)[0]
        f = pkg.sci_fista_tv if algo == "fista" else pkg.sci_gap_tv
        return f(yd, bits, B, tv, 0.05, 6, 10, **kw)[0]

    ref = solve()
    got = solve(fuse_k="tuned")
    assert torch.equal(got, ref)
    entries = json.loads(path.read_text())
    (key, e), = entries.items()
    assert f"|{algo}|{tv}|200x330x{B}|S10|f32|fgp|launch" in key
    assert [e["fuse_k"], e["tile"]] in e["candidates"] and len(e["ms"]) == len(e["candidates"])
    assert torch.equal(solve(fuse_k="tuned"), ref)  # cache hit


def test_tuned_batch_is_bitwise_the_default_batch(pkg, monkeypatch, tmp_path):
    path = tmp_path / "fuse.json"
    monkeypatch.setenv("SCI_TUNE_CACHE", str(path))
    sizes = [(64, 96, 8), (37, 70, 10), (48, 40, 24), (130, 70, 8)]
    ys, bits = [], []
    for k, (nx, ny, B) in enumerate(sizes):
        case, y = make_problem(nx, ny, B, 500 + k, sigma=0.01)
        ys.append(to_dev(y))
        bits.append(pkg.sci_masks_pack(to_dev(case.masks)))
    batch = pkg.Batch(ys, bits, [s[2] for s in sizes])
    cands = tune.batch_fuse_candidates("vtv", batch.Bs, 10)
    best, ms = pkg.sci_tune_fuse_batched(batch, "vtv", 0.05, 10, cands, storage="f16", reps=2)
    assert best in cands and all(np.isfinite(m) and m > 0 for m in ms)
    # FP32 storage: the carried duals are exact, so every depth gives the same bits
    xs, _ = pkg.sci_gap_tv_batched(batch, "vtv", 0.05, 4, 10)
    ref = [x.clone() for x in xs]
    xs, _ = pkg.sci_gap_tv_batched(batch, "vtv", 0.05, 4, 10, fuse_k="tuned")
    for a, b in zip(xs, ref):
        assert torch.equal(a, b)
    (key, e), = json.loads(path.read_text()).items()
    assert "|batched|vtv|" in key and "|S10|f32|fgp" in key
    with pytest.raises(ValueError):
        pkg.sci_gap_tv_batched(batch, "vtv", 0.05, 4, 10, fuse_k="tuned", init=False)


@pytest.mark.parametrize("algo", ["gap", "admm"])
@pytest.mark.parametrize("tv,B", [("atv", 3), ("itv2d", 2), ("vtv", 8), ("vtv", 10)])
def test_every_tile_class_is_bitwise_the_default(pkg, algo, tv, B):
    """With FP32 storage the tile class, like the depth, changes only the
    launch shape: every class that fits gives the default solve's bits."""
    nx, ny = 150, 210
    case, y = make_problem(nx, ny, B, 300 + B, sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))

    def solve(tile, k):
        if algo == "gap":
            return pkg.sci_gap_tv(to_dev(y), bits, B, tv, 0.05, 3, 7, tile=tile, fuse_k=k)[0].cpu().numpy()
        return pkg.sci_admm_tv(to_dev(y), bits, B, tv, 0.05, 0.01, 3, 7, tile=tile, fuse_k=k)[0].cpu().numpy()

    ref = solve(0, 0)
    for t in pkg.sci_tile_classes(tv, B):
        for k in (0, 2, 7):
            np.testing.assert_array_equal(solve(t, k), ref, err_msg=f"tile={t}, fuse_k={k}")


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("tv,dual", [("atv", "fgp"), ("itv2d", "fgp"), ("atv", "clip")])
def test_one_frame_tile_layouts_agree_bitwise(pkg, storage, tv, dual):
    """The one-frame tiles come in two thread layouts (4 x 4 / 2 x 4 pixel
    blocks and 16- / 8-row column strips) of two sizes.  At one depth they
    round the carried duals at the same points, so even with 16-bit storage
    every layout and size gives the same bits; a 300 x 420 image spans several
    tiles of each with ragged last ones."""
    B, nx, ny = 3, 300, 420
    case, y = make_problem(nx, ny, B, 900, sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    for k in (3, 10):
        outs = {t: pkg.sci_gap_tv(to_dev(y), bits, B, tv, 0.05, 3, 10, tile=t, fuse_k=k, storage=storage,
                                  dual=dual)[1].cpu().numpy() for t in (1, 2, 3, 4)}
        for t in (2, 3, 4):
            np.testing.assert_array_equal(outs[t], outs[1], err_msg=f"tile={t}, fuse_k={k}")


def test_tuned_launch_picks_a_candidate_and_keeps_the_bits(pkg, monkeypatch, tmp_path):
    from paper_2005_08028_gb300 import tune
    monkeypatch.setenv("SCI_TUNE_CACHE", str(tmp_path / "fuse.json"))
    B, nx, ny = 10, 128, 160
    case, y = make_problem(nx, ny, B, 77, sigma=0.01)
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    pair = tune.tuned_launch("gap", to_dev(y), bits, B, "vtv", 0.05, 10)
    assert pair in tune.launch_candidates("vtv", B, 10)
    a = pkg.sci_gap_tv(to_dev(y), bits, B, "vtv", 0.05, 4, 10, fuse_k="tuned")[0].cpu().numpy()
    b = pkg.sci_gap_tv(to_dev(y), bits, B, "vtv", 0.05, 4, 10)[0].cpu().numpy()
    np.testing.assert_array_equal(a, b)
