"""Full-size GPU checks in the benchmark's launch configuration.

512x512x10 (T = 200, S = 10, all six reconstructions): x^(T) and theta^(T)
at 256 seeded voxels and the PSNR against the stored FP64-oracle values
(tests/golden/sci_512x512x10_oracle.json, written by
tests/golden/make_sci_512_golden.py from the oracle alone).

2048x2048x32 GAP-ITV2D (T = 100, S = 10): 16-bit storage with FP32 math
against the FP32 path -- PSNR within 0.1 dB and finite -- and the FP32 path's
own invariants (Phi x = y on every pixel with R > 0, since the data are
noise-free).
"""
import json
import os

import numpy as np
import pytest

import oracle as O
import sci_synth as ss
from gpu_helpers import TOL_F32, lib, make_problem, to_dev, torch

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sci_512x512x10_oracle.json")


@pytest.fixture(scope="module")
def pkg():
    return lib()


@pytest.fixture(scope="module")
def c2(pkg):
    g = json.load(open(GOLDEN))
    cfg = ss.CONFIGS["sci_512x512x10"]
    case, y = make_problem(cfg["nx"], cfg["ny"], cfg["B"], cfg["seed"], mask=cfg["mask"], sigma=cfg["sigma"])
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    return g, cfg, case, to_dev(y), bits


@pytest.mark.parametrize("algo,tv", [(a, t) for a in ("gap", "admm") for t in ("atv", "itv2d", "vtv")])
def test_512x512x10_full_run_against_oracle_samples(pkg, c2, algo, tv):
    g, cfg, case, y, bits = c2
    run = next(r for r in g["runs"] if r["algo"] == algo and r["tv"] == tv)
    pos = np.array(g["sample_positions"])
    if algo == "gap":
        x, th, _ = pkg.sci_gap_tv(y, bits, cfg["B"], tv, cfg["lam"], cfg["outer"], cfg["inner"])
    else:
        x, th, _, _ = pkg.sci_admm_tv(y, bits, cfg["B"], tv, cfg["lam"], cfg["rho"], cfg["outer"], cfg["inner"])
    xs = x.cpu().numpy()[pos[:, 0], pos[:, 1], pos[:, 2]]
    ts = th.cpu().numpy()[pos[:, 0], pos[:, 1], pos[:, 2]]
    assert np.abs(xs - np.array(run["x_samples"])).max() <= TOL_F32
    assert np.abs(ts - np.array(run["theta_samples"])).max() <= TOL_F32
    assert abs(O.psnr(x.cpu().numpy(), case.x_gt) - run["psnr_x"]) <= 0.05


def test_2048x2048x32_reduced_precision_storage(pkg):
    cfg = ss.CONFIGS["gap_itv2d_2048x2048x32"]
    case = ss.make_case(cfg["nx"], cfg["ny"], cfg["B"], cfg["seed"], mask=cfg["mask"], sigma=cfg["sigma"])
    x_gt = to_dev(case.x_gt.astype(np.float32))
    bits = pkg.sci_masks_pack(to_dev(case.masks))
    y = pkg.sci_forward(x_gt, bits)
    N = x_gt.numel()
    res = {}
    for storage in ("f32", "bf16", "f16"):
        x, th, _ = pkg.sci_gap_tv(y, bits, cfg["B"], "itv2d", cfg["lam"], cfg["outer"], cfg["inner"],
                                  storage=storage)
        mse = float(pkg.sci_sqdiff_f64(x, x_gt).item()) / N
        res[storage] = (x, 10 * np.log10(1.0 / mse))
        assert torch.isfinite(x).all()
    for storage in ("bf16", "f16"):
        assert abs(res[storage][1] - res["f32"][1]) <= 0.1, (storage, res[storage][1], res["f32"][1])
    # noise-free: the FP32 output satisfies Phi x = y on covered pixels
    x32 = res["f32"][0]
    yy = pkg.sci_forward(x32, bits)
    R = torch.from_numpy(case.masks.sum(0).astype(np.int32)).to(y.device)
    err = (yy - y).abs()[R > 0].max().item()
    assert err <= 1e-4
