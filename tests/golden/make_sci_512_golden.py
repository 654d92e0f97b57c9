"""Write tests/golden/sci_512x512x10_oracle.json from the FP64 oracle only.

For each of the six reconstructions of the 512x512x10 workload (GAP and
ADMM with rho = 0.01, times ATV / ITV2D / VTV; T = 200 outer, S = 10 inner
FGP updates, lambda = 0.05, one Bernoulli(0.5) mask shifted one pixel per
frame, Gaussian noise sigma = 0.01, seed 2) it stores the PSNR of x^(T)
against the ground truth, ||y - Phi theta^(T)||^2, and x^(T), theta^(T) at
256 seeded voxel positions.  The GPU tests compare against these samples.

Run: python tests/golden/make_sci_512_golden.py   (about 10 minutes on 6 cores)
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
import sci_synth as ss  # noqa: E402

OUT = os.path.join(HERE, "sci_512x512x10_oracle.json")
NSAMPLE = 256


def _inputs():
    cfg = ss.CONFIGS["sci_512x512x10"]
    case = ss.make_case(cfg["nx"], cfg["ny"], cfg["B"], cfg["seed"], mask=cfg["mask"], sigma=cfg["sigma"])
    y = (O.forward(case.x_gt, case.masks) + case.noise).astype(np.float32)
    return cfg, case, y


def sample_positions(B, nx, ny):
    rng = np.random.default_rng(12345)
    return np.stack([rng.integers(0, B, NSAMPLE), rng.integers(0, nx, NSAMPLE),
                     rng.integers(0, ny, NSAMPLE)], axis=1)


def run_one(job):
    algo, tv = job
    cfg, case, y = _inputs()
    t0 = time.time()
    if algo == "gap":
        x, th = O.gap_tv(y, case.masks, cfg["lam"], cfg["outer"], cfg["inner"], tv)
    else:
        x, th, _ = O.admm_tv(y, case.masks, cfg["lam"], cfg["rho"], cfg["outer"], cfg["inner"], tv)
    pos = sample_positions(*x.shape)
    return {
        "algo": algo, "tv": tv, "seconds": time.time() - t0,
        "psnr_x": O.psnr(x, case.x_gt),
        "resid_sq": O.residual_sq(th, y, case.masks),
        "x_samples": [float(x[k, i, j]) for k, i, j in pos],
        "theta_samples": [float(th[k, i, j]) for k, i, j in pos],
    }


def main():
    cfg, _, _ = _inputs()
    jobs = [(a, t) for a in cfg["algo"] for t in cfg["tv"]]
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        results = pool.map(run_one, jobs)
    out = {
        "source": "FP64 oracle (oracle/sci_oracle.py) on the seeded 512x512x10 workload; "
                  "written by tests/golden/make_sci_512_golden.py",
        "config": {k: (list(v) if isinstance(v, tuple) else v) for k, v in cfg.items()},
        "sample_positions": sample_positions(cfg["B"], cfg["nx"], cfg["ny"]).tolist(),
        "runs": results,
    }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print(f"wrote {OUT}")


if __name__ == "__main__":
    main()
