#!/usr/bin/env python3
"""Benchmark: GAP-TV / ADMM-TV video SCI reconstruction throughput on GB300.

Workload (one "step"): the six reconstructions of one 512x512x10 measurement
-- GAP and ADMM (rho = 0.01), each with ATV, ITV2D and VTV FGP priors, T = 200
outer x S = 10 inner iterations, lambda = 0.05, one Bernoulli(0.5) mask
shifted one pixel per frame, Gaussian noise sigma = 0.01 -- on synthetic
videos (textured ellipses over ramps).  Unit: voxel-iterations per second,
one voxel-iteration being one voxel through one outer iteration (projection +
S FGP dual updates + output).

Prints ONE JSON line on rank 0.  `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GAP-TV voxel-iters/s at 512²×10 & batched; PSNR Δ vs FP64 oracle; HBM % peak"
UNIT = "voxel-iters/s"
WORKLOAD = "sci_512x512x10"
COMBOS = [(a, t) for a in ("gap", "admm") for t in ("atv", "itv2d", "vtv")]


def _cfg():
    import sci_synth as ss
    return ss.CONFIGS[WORKLOAD]


def _inputs():
    """Seeded ground truth, masks and noise (no reconstruction arithmetic)."""
    import sci_synth as ss
    c = _cfg()
    return ss.make_case(c["nx"], c["ny"], c["B"], c["seed"], mask=c["mask"], sigma=c["sigma"])


def _workload_desc(c):
    return {
        "workload": f"{WORKLOAD}: GAP + ADMM(rho={c['rho']}) x ATV/ITV2D/VTV-FGP, "
                    f"{c['nx']}x{c['ny']}x{c['B']}, T={c['outer']}, S={c['inner']}, "
                    f"lambda={c['lam']}, Bernoulli(0.5) mask shifted 1 px/frame, sigma={c['sigma']}",
        "nx": c["nx"], "ny": c["ny"], "B": c["B"], "outer_iters": c["outer"],
        "inner_iters": c["inner"], "reconstructions_per_step": len(COMBOS),
    }


# ====================================================================== oracle runs on the host cores

_ORACLE_CASE = None


def _oracle_case():
    """The workload's measurement for the FP64 oracle (built once per process)."""
    global _ORACLE_CASE
    if _ORACLE_CASE is None:
        import oracle as O
        case = _inputs()
        y = (O.forward(case.x_gt, case.masks) + case.noise).astype(np.float32).astype(np.float64)
        _ORACLE_CASE = (case, y)
    return _ORACLE_CASE


def _oracle_job(job):
    """One reconstruction of the workload by the oracle for T outer iterations
    (pool worker); returns its seconds.  job = (algo, tv, T); T = 0 only
    builds the inputs."""
    import oracle as O
    algo, tv, T = job
    c = _cfg()
    case, y = _oracle_case()
    if T == 0:
        return 0.0
    t0 = time.perf_counter()
    if algo == "gap":
        O.gap_tv(y, case.masks, c["lam"], T, c["inner"], tv)
    else:
        O.admm_tv(y, case.masks, c["lam"], c["rho"], T, c["inner"], tv)
    return time.perf_counter() - t0


class OraclePool:
    """The oracle over the host's cores: one process per core (spawned, so a
    process that already holds a CUDA context is never forked), each running
    whole reconstructions; the oracle itself is single-threaded numpy."""

    def __init__(self, procs=None):
        import multiprocessing as mp
        self.procs = max(1, int(procs or os.cpu_count() or 1))
        self.pool = mp.get_context("spawn").Pool(self.procs)
        self.pool.map(_oracle_job, [("gap", "atv", 0)] * self.procs, chunksize=1)  # inputs built, imports done

    def run(self, jobs):
        t0 = time.perf_counter()
        self.pool.map(_oracle_job, jobs, chunksize=1)
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


# ====================================================================== reference arm

def run_reference(args):
    """The FP64 oracle as it stands, on the host cores: each step is the six
    reconstructions of the workload for T = 1 outer iteration, run
    concurrently, one process each."""
    _, rank, _ = dist_env()
    if rank != 0:
        return 0
    c = _cfg()
    N = c["nx"] * c["ny"] * c["B"]
    T_sample = 1
    pool = OraclePool(min(len(COMBOS), os.cpu_count() or 1))
    jobs = [(a, t, T_sample) for a, t in COMBOS]
    for _ in range(args.warmup):
        pool.run(jobs)
    dt = sum(pool.run(jobs) for _ in range(args.steps))
    pool.close()
    units = args.steps * len(COMBOS) * N * T_sample
    value = units / dt
    sample = (f"each step: the 6 reconstructions of the {c['nx']}x{c['ny']}x{c['B']} workload run for "
              f"T={T_sample} outer x S={c['inner']} inner iterations (of T={c['outer']}), concurrently "
              f"on {pool.procs} of the host's {os.cpu_count()} cores")
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _workload_desc(c),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.procs, "kind": "oracle", "sample": sample,
                         "nproc": os.cpu_count()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))
    return 0


# ====================================================================== GPU arm

class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"sci_bench_clocks_{os.getpid()}_gpu{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    """(world size, rank, local rank) from the launcher's environment (1, 0, 0 alone)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def job_time_and_value(t_ms, units_per_rank, world, device=None):
    """Whole-job timing over independent replicas: the slowest rank's time
    (max over ranks, one all_reduce) and the units all ranks processed per
    second of it.  Every rank must call this when world > 1."""
    if world > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_ms = float(tt.item())
    return t_ms, units_per_rank * world / (t_ms * 1e-3)


def run_gpu(args):
    import torch
    import torch.distributed as dist

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2005_08028_gb300 import build as b
    if not os.path.exists(b.LIB_PATH):
        b.build()
    import paper_2005_08028_gb300 as pkg

    c = _cfg()
    B, nx, ny = c["B"], c["nx"], c["ny"]
    N = B * nx * ny
    case = _inputs()
    masks_h = np.ascontiguousarray(case.masks)
    x_gt = torch.from_numpy(case.x_gt.astype(np.float32)).to(dev)
    noise = torch.from_numpy(case.noise.astype(np.float32)).to(dev)
    bits = pkg.sci_masks_pack(torch.from_numpy(masks_h).to(dev))
    y = pkg.sci_forward(x_gt, bits) + noise  # measurement formed on the device by the library

    # persistent per-reconstruction buffers, so each solve replays its cached graph
    bufs = []
    for algo, tv in COMBOS:
        bufs.append(dict(algo=algo, tv=tv, theta=torch.empty((B, nx, ny), device=dev),
                         u=torch.empty((B, nx, ny), device=dev), x=torch.empty((B, nx, ny), device=dev),
                         work=pkg.Workspace(dev)))

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    lanes = _lanes(torch, dev, stream, args.streams)

    def solve_all(yy, bb):
        return _run_six(pkg, torch, lanes, bufs, yy, bb)

    for _ in range(args.warmup):
        solve_all(y, bits)
    torch.cuda.synchronize(dev)

    # ---- timed region: K steps, L2 flushed between steps ----
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    launches = 0
    with Clocks(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            evs[k][0].record(stream)
            launches += solve_all(y, bits)
            evs[k][1].record(stream)
        torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    step_ms = [s.elapsed_time(e) for s, e in evs]
    units_per_rank = args.steps * len(COMBOS) * N * c["outer"]
    t_ms, value = job_time_and_value(sum(step_ms), units_per_rank, world, dev)

    # ---- PSNR of the final reconstructions, against the oracle's (stored) values ----
    psnr = {}
    golden = _golden()
    for bf in bufs:
        mse = float(pkg.sci_sqdiff_f64(bf["x"], x_gt).item()) / N
        p = 10.0 * np.log10(1.0 / mse)
        ref = golden.get((bf["algo"], bf["tv"])) if golden else None
        psnr[f"{bf['algo']}_{bf['tv']}"] = {"gpu_db": round(p, 4),
                                           "oracle_db": None if ref is None else round(ref, 4),
                                           "delta_db": None if ref is None else round(p - ref, 4)}

    # ---- dominant kernel: one temporally blocked FGP launch (k_fgp_fused) per TV form, CUDA events ----
    roof = _roofline(pkg, torch, dev, stream, c, B, nx, ny)

    # ---- batched: 256 mixed-size measurements per call (BF16, FP16 and FP32 storage) ----
    batched = None if args.no_batched else _batched(pkg, torch, dev, stream, flush)

    # ---- the Chambolle TVdenoise box on the same measurement ----
    cham = _chambolle(pkg, torch, dev, stream, flush, c, y, bits, x_gt, psnr)
    fista = _fista(pkg, torch, dev, stream, flush, c, y, bits, x_gt, psnr)
    twist = _twist(pkg, torch, dev, stream, flush, c, y, bits, x_gt, psnr)
    clip = _clip(pkg, torch, dev, stream, flush, c, y, bits, x_gt, psnr)
    warm = _warm_start(pkg, torch, dev, stream, flush, c, y, bits, x_gt, psnr)

    # ---- fuse-depth autotuner on the same measurement (outside every timed region) ----
    tuning = None if args.no_tune else _fuse_tuning(pkg, c, y, bits)

    # ---- precision: GAP-ITV2D on 2048x2048x32 with FP32 / FP16 / BF16 storage ----
    precision = None if args.no_precision else _precision(pkg, torch, dev, stream, flush)
    # ---- error against the FP64 oracle for every storage type (stored oracle runs) ----
    vs_fp64 = None if args.no_precision else _vs_fp64(pkg, torch, dev)

    # ---- learned prox: trained here, then GAP-TV on 64 measurements of 512x512x10 ----
    learned = None if args.no_learned else _learned(pkg, torch, dev, stream, flush)

    # ---- end to end: host buffers through the public API ----
    e2e = _e2e(pkg, torch, dev, stream, args, c, masks_h, y, bufs, flush, lanes, world)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(_workload_desc(c), l2="flushed between timed steps (256 MiB write)",
                       parallelism=f"replicas x{world} (independent measurements, no collective)",
                       streams=len(lanes),
                       step_ms=[round(s, 3) for s in step_ms],
                       paper_context="paper: ~3 min for 150 iterations of 512x512x10 ITV3D-FGP on an "
                                     "i7 laptop (about 2.2e6 voxel-iters/s; real data, inner iterations "
                                     "not stated)"),
        "psnr": psnr,
        "chambolle": cham,
        "fista": fista,
        "twist": twist,
        "clip": clip,
        "warm_start": warm,
        "precision_vs_fp64": vs_fp64,
        "fuse_tuning": tuning,
        "batched": batched,
        "precision": precision,
        "learned": learned,
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = _cpu_baseline(c, case)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()
    return 0


def _lanes(torch, dev, stream, n):
    """The streams the six reconstructions of a step are spread over: the
    launching stream first, then n - 1 more."""
    return [stream] + [torch.cuda.Stream(dev) for _ in range(max(1, n) - 1)]


def _run_six(pkg, torch, lanes, bufs, yy, bb, outs_h=None):
    """One step: reconstruction i runs on stream i mod len(lanes) (each has
    its own buffers and workspace), after everything already queued on the
    launching stream, which then waits for all of them.  With outs_h, each
    x^(T) is copied to its pinned host buffer on its reconstruction's stream.
    Returns the number of kernels launched."""
    main = lanes[0]
    for s in lanes[1:]:
        s.wait_stream(main)
    n = 0
    for i, bf in enumerate(bufs):
        with torch.cuda.stream(lanes[i % len(lanes)]):
            _solve(pkg, bf, yy, bb)
            n += pkg.sci_last_solve_launches()
            if outs_h is not None:
                outs_h[i].copy_(bf["x"], non_blocking=True)
    for s in lanes[1:]:
        main.wait_stream(s)
    return n


def _solve(pkg, bf, y, bits):
    c = _cfg()
    if bf["algo"] == "gap":
        pkg.sci_gap_tv(y, bits, c["B"], bf["tv"], c["lam"], c["outer"], c["inner"], x_out=bf["x"],
                       work=bf["work"], theta=bf["theta"], init=True)
    else:
        pkg.sci_admm_tv(y, bits, c["B"], bf["tv"], c["lam"], c["rho"], c["outer"], c["inner"], x_out=bf["x"],
                        work=bf["work"], theta=bf["theta"], u=bf["u"], init=True)


def _golden():
    path = os.path.join(ROOT, "tests", "golden", "sci_512x512x10_oracle.json")
    if not os.path.exists(path):
        return None
    g = json.load(open(path))
    return {(r["algo"], r["tv"]): r["psnr_x"] for r in g["runs"]}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        p = json.load(open(path))
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


ALU_OPS_PER_UPDATE = 20  # FP32 operations per voxel per FGP dual update (FMA = 1)

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per k_fgp_fused
# launch of the roofline case below (one prox launch on 10 x 512 x 512 FP32,
# default updates per launch), from one ncu capture of the current kernel
# (its summary is kept under profiles/); empty when the kernel has changed
# since the capture.  The launch must move at least the 10.49 MB input; its
# 10.49 MB output stays in L2.
NCU_DRAM_BYTES_PER_LAUNCH = {"atv": 10558464, "itv2d": 10557952, "vtv": 10586112}


def _alu_peak():
    """FP32 lane-operations per second: 152 SMs x 128 FP32 lanes x the max SM clock."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    mhz = 2070.0
    if os.path.exists(path):
        mhz = float(json.load(open(path)).get("sm_max_mhz", mhz))
    return 152 * 128 * mhz * 1e6


def _roofline(pkg, torch, dev, stream, c, B, nx, ny):
    """The dominant kernel, the temporally blocked FGP launch (k_fgp_fused):
    sci_tv_prox with S equal to the solver's updates per launch is exactly one
    such launch; it is timed with CUDA events for each TV form."""
    N = B * nx * ny
    x = torch.rand((B, nx, ny), device=dev)
    work = pkg.Workspace(dev)
    per_tv, ops, ms_total, traffic = {}, 0.0, 0.0, []
    for tv in ("atv", "itv2d", "vtv"):
        K = pkg.sci_fused_updates(tv, B, c["inner"], 0)
        if K <= 0:
            continue
        for _ in range(3):
            pkg.sci_tv_prox(x, tv, c["lam"], K, work=work)
        reps = 20
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            pkg.sci_tv_prox(x, tv, c["lam"], K, work=work)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / reps
        per_tv[tv] = {"updates_per_launch": K, "launch_ms": round(ms, 5),
                      "frac": round(ALU_OPS_PER_UPDATE * N * K / (ms * 1e-3) / _alu_peak(), 4),
                      "dram_bytes_ncu": NCU_DRAM_BYTES_PER_LAUNCH.get(tv)}
        traffic.append(NCU_DRAM_BYTES_PER_LAUNCH.get(tv))
        ops += ALU_OPS_PER_UPDATE * N * K
        ms_total += ms
    achieved = ops / (ms_total * 1e-3) / 1e12
    peak = _alu_peak() / 1e12
    return {"kernel": "k_fgp_fused (temporally blocked FGP dual updates)", "bound": "alu",
            "achieved": round(achieved, 3), "peak": round(peak, 3),
            "peak_kind": "derived: 152 SMs x 128 FP32 lanes x max SM clock", "unit": "T FP32-op/s",
            "frac": round(achieved / peak, 4),
            "traffic": (round(sum(traffic) / len(traffic)) if traffic and None not in traffic
                        and (B, nx, ny) == (10, 512, 512) else None),
            "traffic_unit": "bytes per launch (mean over the TV forms, ncu)",
            "alg_ops_per_voxel_update": ALU_OPS_PER_UPDATE, "per_tv": per_tv}


def _batched(pkg, torch, dev, stream, flush):
    """The batched workload: 256 measurements whose sizes are drawn uniformly
    from {128^2 x 8, 256^2 x 8, 512^2 x 10, 1024^2 x 24}, VTV, T = 100,
    S = 5, Bernoulli(0.5) masks, sigma = 0.01, solved in one sci_gap_tv_batched
    call (one CUDA graph).  One ground-truth video per size class (seeded);
    masks and noise differ per measurement.  The fused depth comes from the
    launch-shape autotuner (tune.tuned_batch_fuse: probe solves timed in the
    batch's own buffers on first use, then its JSON cache).  Timed once per
    storage type after one warm-up call, L2 flushed before.  The workload's configured
    storage is BF16 (the section's value); FP16 and FP32 run beside it, and
    each 16-bit format's mean PSNR change against FP32 is checked against the
    0.1 dB gate and reported whether it passes or not."""
    import sci_synth as ss
    bc = ss.CONFIGS["batched_vtv_256"]
    sizes = ss.batch_sizes(bc["count"], bc["sizes"], bc["seed"])
    gts = {}
    for k, (nx, ny, B) in enumerate(bc["sizes"]):
        v = ss.video(nx, ny, B, np.random.default_rng(np.random.SeedSequence(bc["seed"]).spawn(5 + k)[-1]))
        gts[(nx, ny, B)] = torch.from_numpy(v.astype(np.float32)).to(dev)
    ys, bits = [], []
    for m, (nx, ny, B) in enumerate(sizes):
        msk, g = ss.masks_and_noise_torch(nx, ny, B, bc["sigma"], 1000 * bc["seed"] + m, dev)
        bb = pkg.sci_masks_pack(msk, check=False)
        ys.append(pkg.sci_forward(gts[(nx, ny, B)], bb) + g)
        bits.append(bb)
        del msk
    voxels = sum(nx * ny * B for nx, ny, B in sizes)
    out = {"workload": f"batched_vtv_256: {len(sizes)} measurements from {list(bc['sizes'])}, VTV, "
                       f"T={bc['outer']}, S={bc['inner']}, lambda={bc['lam']}, sigma={bc['sigma']}",
           "voxels": voxels, "counts": {f"{a}x{b}x{c}": sizes.count((a, b, c)) for a, b, c in bc["sizes"]}}
    from paper_2005_08028_gb300 import tune
    for storage in ("bf16", "f16", "f32"):
        batch = pkg.Batch(ys, bits, [s[2] for s in sizes])
        # the fused depth from the autotuner (timed once per GPU, batch, S and
        # storage, then cached), before the warm-up call
        k = tune.tuned_batch_fuse(batch, "vtv", bc["lam"], bc["inner"], storage=storage)
        pkg.sci_gap_tv_batched(batch, "vtv", bc["lam"], bc["outer"], bc["inner"], storage=storage, fuse_k=k)
        torch.cuda.synchronize(dev)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pkg.sci_gap_tv_batched(batch, "vtv", bc["lam"], bc["outer"], bc["inner"], storage=storage, fuse_k=k)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        ps = []
        for x, (nx, ny, B) in zip(batch.x_outs, sizes):
            mse = float(pkg.sci_sqdiff_f64(x, gts[(nx, ny, B)]).item()) / (nx * ny * B)
            ps.append(10.0 * np.log10(1.0 / mse))
        out[storage] = {"value": voxels * bc["outer"] / (ms * 1e-3), "unit": UNIT, "ms": round(ms, 2),
                        "mean_psnr_db": round(float(np.mean(ps)), 4), "tuned_fuse_k": int(k),
                        "gpu_launches": pkg.sci_last_batch_launches()}
        del batch
        torch.cuda.empty_cache()
    out["configured_storage"] = "bf16"
    out["value"] = out["bf16"]["value"]
    out["unit"] = UNIT
    for st in ("bf16", "f16"):
        d = round(out[st]["mean_psnr_db"] - out["f32"]["mean_psnr_db"], 4)
        out[f"psnr_delta_{st}_vs_f32_db"] = d
        out[f"gate_0p1db_{st}"] = "pass" if abs(d) <= 0.1 else f"miss ({d:+.3f} dB)"
    return out


def _vs_fp64(pkg, torch, dev):
    """Error against the FP64 oracle for 16-bit and FP32 storage, from
    tests/golden/precision_oracle.json (written by the oracle alone): the
    512x512x32 instance of the precision workload (GAP-ITV2D, T = 100, S = 10,
    through sci_gap_tv) and two measurements of each size class of the batched
    workload (VTV, T = 100, S = 5, through one sci_gap_tv_batched call).  Per
    storage: max-abs and RMS of x^(T) minus the oracle's at the stored sample
    voxels, and the whole-cube PSNR change against the oracle's."""
    import sci_synth as ss
    path = os.path.join(ROOT, "tests", "golden", "precision_oracle.json")
    if not os.path.exists(path):
        return None
    runs = json.load(open(path))["runs"]
    cases = {}
    for r in runs:
        case = ss.make_case(r["nx"], r["ny"], r["B"], r["seed"], sigma=r["sigma"])
        import oracle as O
        y = (O.forward(case.x_gt, case.masks) + case.noise).astype(np.float32)
        cases[r["name"]] = (torch.from_numpy(y).to(dev), pkg.sci_masks_pack(torch.from_numpy(case.masks).to(dev)),
                            torch.from_numpy(case.x_gt.astype(np.float32)).to(dev))
        del case

    def errs(x, r):
        pos = np.asarray(r["positions"])
        xs = x[pos[:, 0], pos[:, 1], pos[:, 2]].double().cpu().numpy()
        d = xs - np.asarray(r["x_samples"])
        gt = cases[r["name"]][2]
        mse = float(pkg.sci_sqdiff_f64(x, gt).item()) / x.numel()
        return float(np.abs(d).max()), d, 10.0 * np.log10(1.0 / mse) - r["psnr_x"]

    out = {"source": "tests/golden/precision_oracle.json (FP64 oracle)", "sampled_voxels_per_run": len(runs[0]["positions"])}
    one = [r for r in runs if r["tv"] == "itv2d"]
    strata = [r for r in runs if r["tv"] == "vtv"]
    for storage in ("f32", "f16", "bf16"):
        sec = {}
        for r in one:
            y, bits, _ = cases[r["name"]]
            x, _, _ = pkg.sci_gap_tv(y, bits, r["B"], "itv2d", r["lam"], r["T"], r["S"], storage=storage)
            mx, d, dp = errs(x, r)
            sec[r["name"]] = {"max_abs": round(mx, 6), "rms": float(f"{np.sqrt(np.mean(d * d)):.3e}"),
                              "dpsnr_vs_fp64_db": round(dp, 4)}
        batch = pkg.Batch([cases[r["name"]][0] for r in strata], [cases[r["name"]][1] for r in strata],
                          [r["B"] for r in strata])
        r0 = strata[0]
        pkg.sci_gap_tv_batched(batch, "vtv", r0["lam"], r0["T"], r0["S"], storage=storage)
        ds, mxs, dps = [], [], {}
        for r, x in zip(strata, batch.x_outs):
            mx, d, dp = errs(x, r)
            ds.append(d)
            mxs.append(mx)
            dps[r["name"]] = round(dp, 4)
        dd = np.concatenate(ds)
        sec["batched_vtv_strata"] = {"max_abs": round(max(mxs), 6), "rms": float(f"{np.sqrt(np.mean(dd * dd)):.3e}"),
                                     "max_abs_dpsnr_vs_fp64_db": round(max(abs(v) for v in dps.values()), 4),
                                     "dpsnr_vs_fp64_db": dps}
        out[storage] = sec
        del batch
    del cases
    torch.cuda.empty_cache()
    return out


def _warm_start(pkg, torch, dev, stream, flush, c, y, bits, x_gt, psnr_cold):
    """The dual warm start (Algorithm 1 initialises w once, before the outer
    loop) in GAP-TV on the 512x512x10 measurement, T = 200: S = 2 dual
    updates per TVdenoise carried from call to call, against the cold start
    with S = 2 and the step's cold S = 10 (PSNR from the timed step).  One timed
    solve each after a warm-up, L2 flushed before."""
    B, nx, ny = c["B"], c["nx"], c["ny"]
    N = B * nx * ny
    theta = torch.empty((B, nx, ny), device=dev)
    x = torch.empty_like(theta)
    work = pkg.Workspace(dev)
    out = {"workload": f"GAP-TV, {nx}x{ny}x{B}, T={c['outer']}, lambda={c['lam']}: warm-started S=2 against "
                       f"cold S=2 and cold S={c['inner']}"}
    for tv in ("atv", "itv2d", "vtv"):
        row = {}
        for label, S, warm in (("warm_S2", 2, True), ("cold_S2", 2, False)):
            def run():
                pkg.sci_gap_tv(y, bits, B, tv, c["lam"], c["outer"], S, theta=theta, x_out=x, init=True, work=work,
                               warm_start=warm)
            run()
            torch.cuda.synchronize(dev)
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1)
            mse = float(pkg.sci_sqdiff_f64(x, x_gt).item()) / N
            row[label] = {"value": N * c["outer"] / (ms * 1e-3), "unit": UNIT, "ms": round(ms, 2),
                          "psnr_db": round(10.0 * np.log10(1.0 / mse), 4)}
        row["cold_S10_psnr_db"] = psnr_cold.get(f"gap_{tv}", {}).get("gpu_db")
        if row["cold_S10_psnr_db"] is not None:
            row["warm_S2_minus_cold_S10_db"] = round(row["warm_S2"]["psnr_db"] - row["cold_S10_psnr_db"], 4)
        out[tv] = row
    return out


def _twist(pkg, torch, dev, stream, flush, c, y, bits, x_gt, psnr_gap):
    """TwIST-TV (Sec. 2.2; steps on Phi / sqrt(L), alpha and beta from the
    eigenvalue bounds of the normalised Phi^T Phi, FGP box) on the 512x512x10
    measurement, T = 200, S = 10: one timed solve per TV form after a warm-up,
    L2 flushed before; PSNR beside GAP-TV's."""
    B, nx, ny = c["B"], c["nx"], c["ny"]
    N = B * nx * ny
    theta = torch.empty((B, nx, ny), device=dev)
    x = torch.empty_like(theta)
    work = pkg.Workspace(dev)
    out = {"workload": f"TwIST-TV, {nx}x{ny}x{B}, T={c['outer']}, S={c['inner']}, lambda={c['lam']}"}
    for tv in ("atv", "itv2d", "vtv"):
        def run():
            pkg.sci_twist_tv(y, bits, B, tv, c["lam"], c["outer"], c["inner"], theta=theta, x_out=x, init=True,
                             work=work)
        run()
        torch.cuda.synchronize(dev)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        mse = float(pkg.sci_sqdiff_f64(x, x_gt).item()) / N
        out[tv] = {"value": N * c["outer"] / (ms * 1e-3), "unit": UNIT, "ms": round(ms, 2),
                   "psnr_db": round(10.0 * np.log10(1.0 / mse), 4),
                   "psnr_gap_db": psnr_gap.get(f"gap_{tv}", {}).get("gpu_db")}
    return out


def _clip(pkg, torch, dev, stream, flush, c, y, bits, x_gt, psnr_fgp):
    """The ATV-Clip box (Algorithm 1; threshold lambda, step 1/4) in GAP-TV and
    ADMM-TV on the 512x512x10 measurement, T = 200, S = 10: one timed solve
    each after a warm-up, L2 flushed before; PSNR beside the FGP box's."""
    B, nx, ny = c["B"], c["nx"], c["ny"]
    N = B * nx * ny
    theta = torch.empty((B, nx, ny), device=dev)
    u = torch.empty_like(theta)
    x = torch.empty_like(theta)
    work = pkg.Workspace(dev)
    out = {"workload": f"ATV-Clip box, {nx}x{ny}x{B}, T={c['outer']}, S={c['inner']}, lambda={c['lam']}"}
    for algo in ("gap", "admm"):
        def run():
            if algo == "gap":
                pkg.sci_gap_tv(y, bits, B, "atv", c["lam"], c["outer"], c["inner"], theta=theta, x_out=x,
                               init=True, work=work, dual="clip")
            else:
                pkg.sci_admm_tv(y, bits, B, "atv", c["lam"], c["rho"], c["outer"], c["inner"], theta=theta, u=u,
                                x_out=x, init=True, work=work, dual="clip")
        run()
        torch.cuda.synchronize(dev)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        mse = float(pkg.sci_sqdiff_f64(x, x_gt).item()) / N
        out[algo] = {"value": N * c["outer"] / (ms * 1e-3), "unit": UNIT, "ms": round(ms, 2),
                     "psnr_db": round(10.0 * np.log10(1.0 / mse), 4),
                     "psnr_fgp_db": psnr_fgp.get(f"{algo}_atv", {}).get("gpu_db")}
    return out


def _chambolle(pkg, torch, dev, stream, flush, c, y, bits, x_gt, psnr_fgp):
    """The Chambolle TVdenoise box (Algorithm 1, ATV-Cham; ITV2D / ITV3D
    norms) in GAP-TV on the same 512x512x10 measurement, T = 200, S = 10: one
    timed solve per TV form after a warm-up, L2 flushed before.  PSNR beside
    the FGP box's (the comparison of the paper's Table 1 columns)."""
    B, nx, ny = c["B"], c["nx"], c["ny"]
    N = B * nx * ny
    theta = torch.empty((B, nx, ny), device=dev)
    x = torch.empty_like(theta)
    work = pkg.Workspace(dev)
    out = {"workload": f"GAP-TV with the Chambolle box, {nx}x{ny}x{B}, T={c['outer']}, S={c['inner']}, "
                       f"lambda={c['lam']}"}
    for tv in ("atv", "itv2d", "vtv"):
        def run():
            pkg.sci_gap_tv(y, bits, B, tv, c["lam"], c["outer"], c["inner"], theta=theta, x_out=x, init=True,
                           work=work, dual="cham")
        run()
        torch.cuda.synchronize(dev)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        mse = float(pkg.sci_sqdiff_f64(x, x_gt).item()) / N
        out[tv] = {"value": N * c["outer"] / (ms * 1e-3), "unit": UNIT, "ms": round(ms, 2),
                   "psnr_db": round(10.0 * np.log10(1.0 / mse), 4),
                   "psnr_fgp_db": psnr_fgp.get(f"gap_{tv}", {}).get("gpu_db")}
    return out


def _fista(pkg, torch, dev, stream, flush, c, y, bits, x_gt, psnr_gap):
    """FISTA-TV (Sec. 2.2; L = max R, the same lambda as GAP, FGP box) on the
    same 512x512x10 measurement, T = 200, S = 10: one timed solve per TV form
    after a warm-up, L2 flushed before.  PSNR beside GAP-TV's (the framework
    rows of the paper's Table 1)."""
    B, nx, ny = c["B"], c["nx"], c["ny"]
    N = B * nx * ny
    theta = torch.empty((B, nx, ny), device=dev)
    x = torch.empty_like(theta)
    work = pkg.Workspace(dev)
    out = {"workload": f"FISTA-TV, {nx}x{ny}x{B}, T={c['outer']}, S={c['inner']}, lambda={c['lam']}"}
    for tv in ("atv", "itv2d", "vtv"):
        def run():
            pkg.sci_fista_tv(y, bits, B, tv, c["lam"], c["outer"], c["inner"], theta=theta, x_out=x, init=True,
                             work=work)
        run()
        torch.cuda.synchronize(dev)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        mse = float(pkg.sci_sqdiff_f64(x, x_gt).item()) / N
        out[tv] = {"value": N * c["outer"] / (ms * 1e-3), "unit": UNIT, "ms": round(ms, 2),
                   "psnr_db": round(10.0 * np.log10(1.0 / mse), 4),
                   "psnr_gap_db": psnr_gap.get(f"gap_{tv}", {}).get("gpu_db")}
    return out


def _fuse_tuning(pkg, c, y, bits):
    """sci_tune_launch on each of the six reconstructions: every (fuse depth,
    tile class) pair the library can run (4 outer iterations per probe, median
    of 5 CUDA-event timings), the chosen pair and the library default (0, 0).
    A failure is reported in the section."""
    from paper_2005_08028_gb300 import tune
    out = {"probe": "4 outer iterations, median of 5, ms per probe; keys are 'fuse_k@tile'"}
    try:
        for algo, tv in COMBOS:
            cands = tune.launch_candidates(tv, c["B"], c["inner"])
            best, ms = pkg.sci_tune_launch(algo, y, bits, c["B"], tv, c["lam"], c["inner"], cands,
                                           rho=c["rho"] if algo == "admm" else 0.0, probe_iters=4, reps=5)
            out[f"{algo}_{tv}"] = {"best": list(cands[best]), "default": [0, 0],
                                   "default_depth": pkg.sci_fused_updates(tv, c["B"], c["inner"], 0),
                                   "ms": {f"{k}@{t}": round(m, 4) for (k, t), m in zip(cands, ms)}}
    except Exception as e:  # noqa: BLE001 -- the section reports its own failure
        out["error"] = f"{type(e).__name__}: {e}"
    return out


def _precision(pkg, torch, dev, stream, flush):
    """GAP-ITV2D on 2048x2048x32 (Bernoulli(0.5) masks, noise-free), T = 100,
    S = 10, with the solver's fields stored as FP32, FP16 and BF16 (FP32
    arithmetic throughout).  Timed once per storage after a warm-up call; every
    field (512 MiB in FP32) is larger than L2.  Reports voxel-iters/s, PSNR
    against the ground truth and its change against FP32, and the whole solve's
    two roofline fractions.  Bytes: what the method must move per voxel and
    outer iteration, i.e. read and write theta (2 x the field width), y
    (4 / B bytes) and the mask word (4 / B), against the measured HBM rate.
    Operations: 20 FP32 operations per voxel per dual update plus 3 for the
    projection, against the derived FP32 ALU peak."""
    import sci_synth as ss
    cfg = ss.CONFIGS["gap_itv2d_2048x2048x32"]
    nx, ny, B, T, S = cfg["nx"], cfg["ny"], cfg["B"], cfg["outer"], cfg["inner"]
    case = ss.make_case(nx, ny, B, cfg["seed"], mask=cfg["mask"], sigma=cfg["sigma"])
    x_gt = torch.from_numpy(case.x_gt.astype(np.float32)).to(dev)
    bits = pkg.sci_masks_pack(torch.from_numpy(case.masks).to(dev))
    del case
    y = pkg.sci_forward(x_gt, bits)
    N = B * nx * ny
    hbm, hbm_kind = _peaks()
    alu = _alu_peak()
    out = {"workload": f"gap_itv2d_2048x2048x32: GAP-ITV2D, {nx}x{ny}x{B}, T={T}, S={S}, "
                       f"lambda={cfg['lam']}, Bernoulli(0.5) masks, noise-free"}
    theta = torch.empty((B, nx, ny), device=dev)
    x = torch.empty_like(theta)
    work = pkg.Workspace(dev)
    for storage in ("f32", "f16", "bf16"):
        def run():
            pkg.sci_gap_tv(y, bits, B, "itv2d", cfg["lam"], T, S, theta=theta, x_out=x, init=True, work=work,
                           storage=storage)
        run()
        torch.cuda.synchronize(dev)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        mse = float(pkg.sci_sqdiff_f64(x, x_gt).item()) / N
        width = 4 if storage == "f32" else 2
        bytes_alg = (2 * width + 8.0 / B) * N * T
        ops_alg = (ALU_OPS_PER_UPDATE * S + 3) * N * T
        out[storage] = {"value": N * T / (ms * 1e-3), "unit": UNIT, "ms": round(ms, 2),
                        "psnr_db": round(10.0 * np.log10(1.0 / mse), 4),
                        "hbm_frac": round(bytes_alg / (ms * 1e-3) / (hbm * 1e9), 4),
                        "alu_frac": round(ops_alg / (ms * 1e-3) / alu, 4)}
    for storage in ("f16", "bf16"):
        out[storage]["delta_db_vs_f32"] = round(out[storage]["psnr_db"] - out["f32"]["psnr_db"], 4)
    out["peaks"] = {"hbm_gbs": hbm, "hbm_kind": hbm_kind, "alu_tops": round(alu / 1e12, 3)}
    del theta, x, work, y, x_gt, bits
    torch.cuda.empty_cache()
    return out


def _learned(pkg, torch, dev, stream, flush):
    """Learned prox replacing S = 10 VTV-FGP updates inside GAP-TV.

    Training: 20480 (x, FGP_10(x)) pairs of 64x64x8 patches (the config's
    20k) cut from plain GAP-TV runs on seeded 256x256x8 measurements stopped
    at random outer iterations in [1, 50], plus 512 held out; Adam, 8 epochs
    of batch 32.  Test: 64 measurements of 512x512x10 (Bernoulli(0.5) masks,
    sigma = 0.01), T = 50 outer iterations with the learned prox and a
    residual check every 10 iterations against the plain method's residual
    curve (calibrated on 8 held-out measurements), falling back to plain FGP
    where it is exceeded by more than 5%.  Compared with plain FP32 GAP-TV
    (VTV, S = 10) on the same 64 measurements.  The tensor-core convolution's
    own throughput is measured on the test batch's activations."""
    import paper_2005_08028_gb300.lprox_train as LT
    import sci_synth as ss
    lam, S, T, every = 0.05, 10, 50, 10
    t0 = time.perf_counter()
    n_train, n_held = 20480, 512
    X, Y = LT.make_pairs(n_train + n_held, seed=50, size=(256, 256, 8))
    net = pkg.LearnedProx(params=LT.init_params(seed=1))
    hist = LT.train(net, X[:n_train], Y[:n_train], epochs=8, batch=32, lr=1e-3)
    pred = net.apply(X[n_train:])
    mse_net = float(((pred - Y[n_train:]) ** 2).mean())
    mse_id = float(((X[n_train:] - Y[n_train:]) ** 2).mean())
    torch.cuda.synchronize(dev)
    train_s = time.perf_counter() - t0
    del X, Y, pred

    def meas(count, seed0):
        ys, bs, gts = [], [], []
        for k in range(count):
            c = ss.make_case(512, 512, 10, seed0 + k, sigma=0.01)
            bb = pkg.sci_masks_pack(torch.from_numpy(c.masks).to(dev))
            xg = torch.from_numpy(c.x_gt.astype(np.float32)).to(dev)
            ys.append(pkg.sci_forward(xg, bb) + torch.from_numpy(c.noise.astype(np.float32)).to(dev))
            bs.append(bb)
            gts.append(xg)
        return torch.stack(ys), torch.stack(bs), gts

    # calibration: the plain method's residual every 10 iterations on held-out measurements
    yc, bc, _ = meas(8, 52000)
    curves = []
    for k in range(8):
        _, _, r = pkg.sci_gap_tv(yc[k].contiguous(), bc[k].contiguous(), 10, "vtv", lam, T, S, resid_every=every)
        curves.append(r.cpu().numpy())
    limit = np.mean(curves, axis=0).tolist()
    y, bits, gts = meas(64, 51000)
    N = 64 * 10 * 512 * 512
    work = pkg.Workspace(dev)
    pkg.sci_gap_tv_lprox(net, y[:2], bits[:2], 10, 2, work=work)  # warm-up
    torch.cuda.synchronize(dev)
    flush.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    x_l, _, fell, hist_l = pkg.sci_gap_tv_lprox(net, y, bits, 10, T, check_every=every, resid_limit=limit,
                                                work=work)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_l = e0.elapsed_time(e1)
    # plain FP32 GAP-TV on the same measurements (one solve each, cached graph after the first)
    xs_p = []
    pw = pkg.Workspace(dev)
    th = torch.empty((10, 512, 512), device=dev)
    xo = [torch.empty((10, 512, 512), device=dev) for _ in range(64)]
    pkg.sci_gap_tv(y[0].contiguous(), bits[0].contiguous(), 10, "vtv", lam, T, S, theta=th, init=True,
                   x_out=xo[0], work=pw)
    torch.cuda.synchronize(dev)
    flush.zero_()
    e0.record(stream)
    for k in range(64):
        pkg.sci_gap_tv(y[k].contiguous(), bits[k].contiguous(), 10, "vtv", lam, T, S, theta=th, init=True,
                       x_out=xo[k], work=pw)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_p = e0.elapsed_time(e1)

    def mean_psnr(xs):
        ps = []
        for x, g in zip(xs, gts):
            mse = float(pkg.sci_sqdiff_f64(x.contiguous(), g).item()) / g.numel()
            ps.append(10.0 * np.log10(1.0 / mse))
        return float(np.mean(ps))

    p_l, p_p = mean_psnr([x_l[k] for k in range(64)]), mean_psnr(xo)
    # The fallback rule's behaviour: plain GAP-TV's own residual curves on the
    # same 64 measurements (untimed), against the calibration band, and the
    # learned run's residual over plain's at each checkpoint.
    curves_t = []
    for k in range(64):
        _, _, r = pkg.sci_gap_tv(y[k].contiguous(), bits[k].contiguous(), 10, "vtv", lam, T, S, resid_every=every,
                                 theta=th, work=pw)
        curves_t.append(r.cpu().numpy())
    Pc, Lc, cal = np.array(curves_t), np.array(hist_l), np.array(curves)
    diag = {"calibration_spread_rel": round(float((cal.std(axis=0) / cal.mean(axis=0)).max()), 4),
            "plain_outside_band": int(((Pc / np.array(limit)) > 1.05).any(axis=1).sum()),
            "learned_outside_band": int(((Lc / np.array(limit)) > 1.05).any(axis=1).sum()),
            "learned_over_plain_residual_mean": [round(float(v), 4) for v in (Lc / Pc).mean(axis=0)],
            "learned_over_plain_residual_max": round(float((Lc / Pc).max()), 4),
            "reading": "the 5% band is narrower than the residual's spread across videos and than the "
                       "learned/plain residual gap on the same measurement at equal PSNR"}
    # tensor-core conv throughput on activations of this size
    act = torch.randn((64, 10, 512, 512, 32), device=dev).to(torch.bfloat16)
    wt = (0.05 * torch.randn((27, 32, 32), device=dev)).to(torch.bfloat16)
    pkg.sci_conv3d_c32_bf16(act[:1], wt)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    out, err = pkg.sci_conv3d_c32_bf16(act, wt)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_c = e0.elapsed_time(e1)
    flops = 2.0 * 27 * 32 * 32 * act[..., 0].numel()
    peak = _bf16_peak()
    del act, out
    return {"workload": "learned_prox_64x512x512x10: VTV, lambda=0.05, T=50, network replaces S=10 FGP "
                        "updates; residual check every 10 iterations, fallback ratio 1.05",
            "train": {"pairs": n_train, "held_out": n_held, "patch": "8x64x64", "epochs": 8, "batch": 32, "seconds": round(train_s, 1),
                      "loss_per_epoch": [float(f"{h:.3e}") for h in hist],
                      "heldout_mse_vs_identity": round(mse_net / mse_id, 4)},
            "learned": {"value": N * T / (ms_l * 1e-3), "unit": UNIT, "ms": round(ms_l, 1),
                        "mean_psnr_db": round(p_l, 4), "fallbacks": int(sum(fell))},
            "fallback_diagnostics": diag,
            "plain_f32": {"value": N * T / (ms_p * 1e-3), "unit": UNIT, "ms": round(ms_p, 1),
                          "mean_psnr_db": round(p_p, 4)},
            "psnr_delta_learned_vs_plain_db": round(p_l - p_p, 4),
            "conv_tc_roofline": {"kernel": "k_conv3d_c32_tc", "bound": "tensor",
                                 "achieved": round(flops / (ms_c * 1e-3) / 1e12, 2), "peak": peak,
                                 "peak_kind": "measured bf16_tflops (burst)", "unit": "TFLOP/s",
                                 "frac": round(flops / (ms_c * 1e-3) / 1e12 / peak, 4),
                                 "err_word": int(err.item())}}


def _bf16_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return float(json.load(open(path))["bf16_tflops"])
    return 1900.0


def _e2e(pkg, torch, dev, stream, args, c, masks_h, y_dev, bufs, flush, lanes, world=1):
    """Same metric through the public API with host inputs/outputs: each step
    copies y and the dense masks from pinned host memory, packs the masks,
    runs the six reconstructions (on the timed step's streams) and copies
    every x^(T) back."""
    B, nx, ny = c["B"], c["nx"], c["ny"]
    N = B * nx * ny
    y_h = y_dev.cpu().pin_memory()
    m_h = torch.from_numpy(masks_h).pin_memory()
    y_d = torch.empty_like(y_dev)
    m_d = torch.empty(m_h.shape, dtype=torch.uint8, device=dev)
    outs_h = [torch.empty((B, nx, ny), dtype=torch.float32).pin_memory() for _ in bufs]

    def step():
        y_d.copy_(y_h, non_blocking=True)
        m_d.copy_(m_h, non_blocking=True)
        bb = pkg.sci_masks_pack(m_d, check=False)
        _run_six(pkg, torch, lanes, bufs, y_d, bb, outs_h)

    step()
    torch.cuda.synchronize(dev)
    total = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        total += e0.elapsed_time(e1)
    units = args.steps * len(bufs) * N * c["outer"]
    _, value = job_time_and_value(total, units, world, dev)
    return {"value": value, "unit": UNIT,
            "h2d_bytes_per_step": int(y_h.numel() * 4 + m_h.numel()),
            "d2h_bytes_per_step": int(len(bufs) * N * 4)}


def _cpu_baseline(c, case):
    """The FP64 oracle on a bounded sample of the workload (T = 1 outer
    iteration per reconstruction), on the host cores: single-threaded (the six
    reconstructions one after another in this process), then on every core
    (nproc processes, each running reconstructions of the workload in turn).
    The all-core rate is the line's value."""
    import oracle as O
    y = (O.forward(case.x_gt, case.masks) + case.noise).astype(np.float32).astype(np.float64)
    N = c["nx"] * c["ny"] * c["B"]
    t0 = time.perf_counter()
    for algo, tv in COMBOS:
        if algo == "gap":
            O.gap_tv(y, case.masks, c["lam"], 1, c["inner"], tv)
        else:
            O.admm_tv(y, case.masks, c["lam"], c["rho"], 1, c["inner"], tv)
    dt1 = time.perf_counter() - t0
    nproc = os.cpu_count() or 1
    pool = OraclePool(nproc)
    jobs = [COMBOS[i % len(COMBOS)] + (1,) for i in range(nproc)]
    dtp = pool.run(jobs)
    pool.close()
    return {"value": len(jobs) * N / dtp, "unit": UNIT, "cores": nproc, "kind": "oracle", "nproc": nproc,
            "sample": f"T=1 outer x S={c['inner']} inner iterations of {len(jobs)} reconstructions of the "
                      f"{c['nx']}x{c['ny']}x{c['B']} workload (the six GAP/ADMM x ATV/ITV2D/VTV in turn), one "
                      f"process per core ({dtp:.1f} s)",
            "single_thread": {"value": len(COMBOS) * N / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"T=1 of each of the 6 reconstructions in turn ({dt1:.1f} s)"}}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["sci", "reference"], default="sci")
    ap.add_argument("--streams", type=int, default=2,
                    help="CUDA streams the six reconstructions of a step are spread over")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 256-measurement batched solve")
    ap.add_argument("--no-learned", action="store_true", help="skip training and running the learned prox")
    ap.add_argument("--no-tune", action="store_true", help="skip the fuse-depth autotuner section")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the 2048x2048x32 FP32 / FP16 / BF16 storage solves")
    ap.add_argument("--kernel-case", choices=["fused", "conv", "lprox", "large", "batched"], default=None,
                    help="run one launch of the dominant kernel per TV form and exit (for profilers)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.kernel_case:
        return run_kernel_case(args)
    return run_gpu(args)


def run_kernel_case(args):
    """fused: one temporally blocked FGP launch per TV form on the 512x512x10
    size.  conv: one tensor-core 32->32 conv over 8 x 10 x 512 x 512 voxels
    (1.3 GB of BF16 activations, larger than L2).  lprox: the learned prox from
    its initial weights, five applies on 8 x 10 x 512 x 512 and five training
    steps on 32 x 8 x 64 x 64 (two of each untimed), timed with CUDA events.
    large: two outer iterations of GAP-ITV2D on the 2048x2048x32 size (512 MiB
    per FP32 field, larger than L2) with FP32, then BF16 storage.  batched: two
    outer iterations of the batched GAP-VTV solve (S = 5, BF16) on eight
    measurements, two of each size class (128x128x8, 256x256x8, 512x512x10,
    1024x1024x24).  The last two draw uniform random videos and Bernoulli(0.5)
    masks on the device: they exist to be profiled, not to be checked."""
    import torch
    from paper_2005_08028_gb300 import build as b
    if not os.path.exists(b.LIB_PATH):
        b.build()
    import paper_2005_08028_gb300 as pkg
    c = _cfg()
    dev = torch.device("cuda")
    if args.kernel_case == "lprox":
        import paper_2005_08028_gb300.lprox_train as LT
        net = pkg.LearnedProx(dev, params=LT.init_params(seed=1, device=dev))
        gen = torch.Generator(device=dev).manual_seed(2)
        x = torch.rand((8, 10, 512, 512), generator=gen, device=dev)
        xt = torch.rand((32, 8, 64, 64), generator=gen, device=dev)
        yt = xt.clone()

        def timed(fn, warm=2, reps=3):
            for _ in range(warm):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        out = {"kernel_case": "lprox", "apply_8x10x512x512_ms": round(timed(lambda: net.apply(x)), 3),
               "train_step_32x8x64x64_ms": round(timed(lambda: net.train_step(xt, yt, 1e-4)), 3)}
        out["ok"] = net.error_word(tuple(x.shape), False) == 0
        print(json.dumps(out))
        return 0 if out["ok"] else 1
    if args.kernel_case == "conv":
        act = torch.randn((8, 10, 512, 512, 32), device=dev).to(torch.bfloat16)
        wt = (0.05 * torch.randn((27, 32, 32), device=dev)).to(torch.bfloat16)
        out, err = pkg.sci_conv3d_c32_bf16(act, wt)
        torch.cuda.synchronize()
        print(json.dumps({"kernel_case": "conv", "ok": int(err.item()) == 0}))
        return 0 if int(err.item()) == 0 else 1
    if args.kernel_case in ("large", "batched"):
        gen = torch.Generator(device=dev).manual_seed(3)

        def measurement(B, nx, ny):
            x = torch.rand((B, nx, ny), generator=gen, device=dev)
            bits = pkg.sci_masks_pack((torch.rand((B, nx, ny), generator=gen, device=dev) < 0.5).to(torch.uint8))
            return pkg.sci_forward(x, bits), bits

        if args.kernel_case == "large":
            B, nx, ny = 32, 2048, 2048
            y, bits = measurement(B, nx, ny)
            theta = torch.empty((B, nx, ny), device=dev)
            work = pkg.Workspace(dev)
            for storage in ("f32", "bf16"):
                pkg.sci_gap_tv(y, bits, B, "itv2d", 0.05, 2, 10, theta=theta, init=True, work=work, storage=storage)
        else:
            ys, bitss, Bs = [], [], []
            for (nx, ny, B) in ((128, 128, 8), (256, 256, 8), (512, 512, 10), (1024, 1024, 24)) * 2:
                y, bits = measurement(B, nx, ny)
                ys.append(y), bitss.append(bits), Bs.append(B)
            batch = pkg.Batch(ys, bitss, Bs)
            pkg.sci_gap_tv_batched(batch, "vtv", 0.05, 2, 5, storage="bf16")
        torch.cuda.synchronize()
        print(json.dumps({"kernel_case": args.kernel_case, "ok": True}))
        return 0
    x = torch.rand((c["B"], c["nx"], c["ny"]), device=dev)
    work = pkg.Workspace(dev)
    for tv in ("atv", "itv2d", "vtv"):
        K = pkg.sci_fused_updates(tv, c["B"], c["inner"], 0)
        pkg.sci_tv_prox(x, tv, c["lam"], K, work=work)
    torch.cuda.synchronize()
    print(json.dumps({"kernel_case": args.kernel_case, "ok": True}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
