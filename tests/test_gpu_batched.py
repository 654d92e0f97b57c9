"""Batched GAP-TV (sci_gap_tv_batched): many measurements of mixed sizes per
launch must reproduce the single-measurement solver exactly (FP32: the fused
tile arithmetic does not depend on the tiling) and the FP64 oracle within
1e-4."""
import pytest

import oracle as O
from gpu_helpers import TOL_F32, lib, make_problem, maxabs, to_dev, torch

pytestmark = pytest.mark.gpu

SIZES = [(37, 70, 3), (64, 96, 8), (20, 30, 10), (16, 40, 24), (1, 1, 1), (130, 70, 5), (48, 33, 16)]


@pytest.fixture(scope="module")
def pkg():
    return lib()


def _batch(pkg, sizes, seed0):
    cases, ys, bits = [], [], []
    for k, (nx, ny, B) in enumerate(sizes):
        case, y = make_problem(nx, ny, B, seed0 + k, sigma=0.01)
        cases.append((case, y))
        ys.append(to_dev(y))
        bits.append(pkg.sci_masks_pack(to_dev(case.masks)))
    return cases, pkg.Batch(ys, bits, [s[2] for s in sizes])


@pytest.mark.parametrize("tv", O.TV_TYPES)
def test_batched_matches_single_and_oracle(pkg, tv):
    cases, batch = _batch(pkg, SIZES, 300)
    T, S = 4, 6
    xs, ths = pkg.sci_gap_tv_batched(batch, tv, 0.05, T, S)
    torch.cuda.synchronize()
    for (case, y), x, th, yd, bb, B in zip(cases, xs, ths, batch.ys, batch.bits, batch.Bs):
        xs1, th1, _ = pkg.sci_gap_tv(yd, bb, B, tv, 0.05, T, S)
        assert torch.equal(x, xs1) and torch.equal(th, th1)
        xr, thr = O.gap_tv(y, case.masks, 0.05, T, S, tv)
        assert maxabs(x, xr) <= TOL_F32 and maxabs(th, thr) <= TOL_F32


def test_batched_graph_replay_and_resume(pkg):
    cases, batch = _batch(pkg, SIZES[:4], 400)
    x1, _ = pkg.sci_gap_tv_batched(batch, "vtv", 0.05, 5, 4)
    x1 = [x.clone() for x in x1]
    x2, _ = pkg.sci_gap_tv_batched(batch, "vtv", 0.05, 5, 4)  # cached graph replay
    for a, b in zip(x1, x2):
        assert torch.equal(a, b)
    # resume: 3 + 2 iterations from the caller's theta equal 5 in one call
    pkg.sci_gap_tv_batched(batch, "vtv", 0.05, 3, 4)
    x3, _ = pkg.sci_gap_tv_batched(batch, "vtv", 0.05, 2, 4, init=False)
    for a, b in zip(x1, x3):
        assert torch.equal(a, b)


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_batched_reduced_precision(pkg, storage):
    cases, batch = _batch(pkg, [(96, 128, 8), (64, 64, 24), (80, 80, 10)], 500)
    xs, _ = pkg.sci_gap_tv_batched(batch, "vtv", 0.05, 15, 5, storage=storage)
    torch.cuda.synchronize()
    for (case, y), x in zip(cases, xs):
        xr, _ = O.gap_tv(y, case.masks, 0.05, 15, 5, "vtv")
        d = abs(O.psnr(x.cpu().numpy(), case.x_gt) - O.psnr(xr, case.x_gt))
        assert d <= 0.1


def test_batched_rejects_vtv_beyond_24_frames(pkg):
    cases, batch = _batch(pkg, [(8, 8, 25)], 600)
    with pytest.raises(pkg.SciError):
        pkg.sci_gap_tv_batched(batch, "vtv", 0.05, 2, 2)
