"""Write tests/golden/precision_oracle.json from the FP64 oracle only.

Two sets of reconstructions, the expected values for the storage-precision
and batched GPU tests (16-bit storage against FP64; the largest batch class
included):

- "gap_itv2d_512x512x32": GAP-TV with ITV2D FGP, T = 100, S = 10,
  lambda = 0.05, i.i.d. Bernoulli(0.5) masks, no noise -- the recipe of the
  2048 x 2048 x 32 precision workload on a 512 x 512 x 32 instance (seed 3);
- "batched_vtv_strata": GAP-TV with VTV FGP, T = 100, S = 5, lambda = 0.05,
  Bernoulli(0.5) masks, sigma = 0.01 -- two measurements of each size class
  of the 256-measurement batched workload (128^2 x 8, 256^2 x 8,
  512^2 x 10, 1024^2 x 24), seeds 4000 + k, drawn on the host.

Each entry stores the PSNR of x^(T) against its ground truth (whole cube,
peak 1) and x^(T) at NSAMPLE seeded voxel positions.

Run: python tests/golden/make_precision_goldens.py   (about 30 minutes on 8 cores)
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

OUT = os.path.join(HERE, "precision_oracle.json")
NSAMPLE = 512
LAM = 0.05

# (name, nx, ny, B, seed, tv, T, S, sigma)
JOBS = [("gap_itv2d_512x512x32", 512, 512, 32, 3, "itv2d", 100, 10, 0.0)]
for cls, (nx, ny, B) in enumerate(((128, 128, 8), (256, 256, 8), (512, 512, 10), (1024, 1024, 24))):
    for rep in range(2):
        JOBS.append((f"vtv_{nx}x{ny}x{B}_{rep}", nx, ny, B, 4000 + 2 * cls + rep, "vtv", 100, 5, 0.01))


def case_of(job):
    """Ground truth, masks and the FP32 measurement of one job (also used by the GPU tests)."""
    _, nx, ny, B, seed, _, _, _, sigma = job
    case = ss.make_case(nx, ny, B, seed, sigma=sigma)
    y = (O.forward(case.x_gt, case.masks) + case.noise).astype(np.float32)
    return case, y


def sample_positions(B, nx, ny, seed):
    rng = np.random.default_rng(777 + seed)
    return np.stack([rng.integers(0, B, NSAMPLE), rng.integers(0, nx, NSAMPLE),
                     rng.integers(0, ny, NSAMPLE)], axis=1)


def run_one(job):
    name, nx, ny, B, seed, tv, T, S, sigma = job
    case, y = case_of(job)
    t0 = time.time()
    x, _ = O.gap_tv(y, case.masks, LAM, T, S, tv)
    pos = sample_positions(B, nx, ny, seed)
    return {"name": name, "nx": nx, "ny": ny, "B": B, "seed": seed, "tv": tv, "T": T, "S": S,
            "sigma": sigma, "lam": LAM, "seconds": round(time.time() - t0, 1),
            "psnr_x": O.psnr(x, case.x_gt),
            "positions": pos.tolist(), "x_samples": [float(x[k, i, j]) for k, i, j in pos]}


def main():
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(JOBS), os.cpu_count() or 4)) as pool:
        runs = pool.map(run_one, JOBS, chunksize=1)
    out = {"about": "FP64 oracle reconstructions for the storage-precision and batched GPU tests "
                    "(written by tests/golden/make_precision_goldens.py)",
           "nsample": NSAMPLE, "runs": runs}
    with open(OUT, "w") as f:
        json.dump(out, f)
    for r in runs:
        print(r["name"], f"{r['psnr_x']:.4f} dB", f"{r['seconds']} s")


if __name__ == "__main__":
    main()
