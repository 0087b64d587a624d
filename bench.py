#!/usr/bin/env python
"""Benchmark of the sorption moment-propagation hot path on one GB300 (or N replicas).

Workload (one "step" = one whole job, every stage of the path on one medium):
  random porous medium 128^3, overlapping solid spheres of radius 6, porosity 0.40, seed 1
  (periodic), uniform body force along x set once so that the mean fluid velocity is 0.01;
    1. geometry prep on the device (node classes, interface bits and offsets),
    2. lb_steady: BGK tau = 1 from rest until max|u(t) - u(t-1)| < 1e-7 (checked every 100),
    3. mp_init: one species, D_b = 0.05, k_a = k_d = 5e-3, FP32 storage, FP64 reductions,
    4. mp_step: 2e4 moment-propagation + sorption steps with Z(t) and D(t) on the device.
Metric: moment-propagation node-species updates per second of the whole job (fluid nodes
x species x MP steps / job time). The LB steps to steady state are reported beside it.
`value` is timed with CUDA events on the launching stream with the medium already on the
device; `e2e` times the same job from a host solid mask to host Z(t)/D(t) arrays.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs an independent replica (no data exchange: the path has none
across jobs); value = all ranks' updates / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = {
    "workload": "random-sphere porous medium 128^3 (R=6, porosity 0.40, seed 1): LB to steady + "
                "2e4 sorption-MP steps, 1 species",
    "lattice": [128, 128, 128],
    "radius": 6,
    "porosity": 0.40,
    "seed": 1,
    "mean_u": 0.01,
    "tau": 1.0,
    "lb_tol": 1e-7,
    "lb_check_every": 100,
    "D_b": 0.05,
    "k_a": 5e-3,
    "k_d": 5e-3,
    "species": 1,
    "mp_steps": 20000,
    "precision": "fp32 storage and arithmetic, fp64 reductions and D(t)",
}
# LB steps to steady state of this workload, measured by the GPU arm (cold start); used only
# to scale the oracle's per-step CPU times to a whole job in the reference arm.
LB_STEPS_ASSUMED = 2000

METRIC = "sorption-MP node-species updates/s (whole job incl. LB to steady)"
UNIT = "node-species updates/s"

# DRAM traffic per launch from ncu (dram__bytes_read.sum + dram__bytes_write.sum), valid only
# while the kernel source hashes to `src_sha`; otherwise reported as null.
TRAFFIC = {
    # ncu --set full, python bench.py --profile, k_step<float,2,1> launch 11 (caches flushed
    # by ncu before the capture, so this is the cold-L2 traffic of one launch). Captured on
    # mp.cu 'cd4af1701d41b82f'; the file changed since only in the flow-packing kernel (64-bit
    # offsets), not in k_step.
    "k_step<float>": {"bytes_per_launch": 48_607_488 + 1_392_640, "src_sha": "450a088ead29ab87"},
    # ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum, python bench.py --profile
    # --scheme direct --variant 2: one persistent launch of 20 steps moved 1299.98 + 93.68 MB;
    # per step (the unit of the roofline entry). Captured on mp_direct.cu 'be2e78e2a2bfa30f';
    # the file changed since only in host code (the tiled variant's block size) and in the
    # several-species kernels (register use, comments), not in this kernel.
    "k_direct_persistent": {"bytes_per_launch": (1_299_980_800 + 93_677_056) // 20, "src_sha": "4588265e46e22840"},
    # the same metrics, python bench.py --profile --scheme direct --variant 4 (one launch per
    # step, link table, blocks of 128; the autotuner's choice when it times within noise of the
    # persistent launch): three launches, 94.13 + 2.56 MB on average. ncu flushes the caches
    # before each captured launch, so this is the cold-L2 traffic of a step (an upper bound;
    # the persistent launch's warm steps move 69.7 MB).
    "k_direct_step": {"bytes_per_launch": (93_998_080 + 94_247_168 + 94_153_984 + 4_150_528 + 1_185_536 + 2_335_744) // 3,
                      "src_sha": "4588265e46e22840"},
    # the same metrics, python bench.py --profile-probe --scheme direct --variant 7: one
    # persistent launch of 20 steps of 192^3 x 4 species (2 830 813 fluid nodes) moved
    # 6175.20 + 2775.19 MB; per step, scaled by the units to the 384^3 x 4 probe
    # (22 649 211 fluid nodes). Captured on mp_direct.cu 'be2e78e2a2bfa30f'; since then the
    # kernel keeps fewer registers live (fewer spills to local memory), same data accesses.
    "k_direct_persistent@probe": {"bytes_per_launch": int((6_175_201_280 + 2_775_187_456) / 20 * 22_649_211 / 2_830_813),
                                  "src_sha": "4588265e46e22840"},
    # ncu --set full, python bench.py --profile-probe --scheme direct --variant 1 (one launch per
    # step, recomputed link terms, blocks of 256): one step of 192^3 x 4 species moved
    # 310.77 + 128.08 MB (cold L2); scaled by the units to the 384^3 x 4 probe. Captured on
    # mp_direct.cu 'be2e78e2a2bfa30f'; the kernel has kept fewer registers live since, same
    # data accesses.
    "k_direct_step@probe": {"bytes_per_launch": int((310_765_824 + 128_075_776) * 22_649_211 / 2_830_813),
                            "src_sha": "4588265e46e22840"},
}


# One-off kernels of one job on this medium, counted in an ncu launch list of the job:
# geometry preparation for the LB and for the MP, cluster labelling (24 sweeps on this
# medium), and the LB and MP initialisation.
JOB_FIXED_LAUNCHES = 42


def _src_sha(name):
    p = os.path.join(ROOT, "paper_1303_2470_gb300", "csrc", name)
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for _, _, flags in rows for n, f in zip(names, flags) if f == "Active"})
        loaded = [r[0] for r in rows]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def aggregate(seconds, units_per_rank, world, dist=None, device=None):
    """Whole-job throughput of N replicas: the slowest rank's time (max over ranks) and all
    ranks' units over it. With world == 1 no collective is used."""
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    slowest = float(t.item())
    return slowest, units_per_rank * world / slowest


# Probe of the MP step on a working set far beyond L2 (the scaled probe of the scope table:
# the benchmark's medium generator at 384^3 with four species), timed inside the default run
# for the HBM roofline. Inputs are synthetic: the seeded drift flow of media.drift_flow (the
# step's cost does not depend on the flow's values) and four species with every p_i > 0.
PROBE = {"lattice": 384, "radius": 6, "porosity": 0.40, "seed": 1, "species": 4, "steps": 200,
         "flow": "media.drift_flow(mean 0.01, noise 0.01, seed 3)", "species_seed": 7,
         "D_b": [0.03, 0.1], "k": [1e-3, 1e-1]}


def run_hbm_probe(mp, peak, peak_kind, scheme_opts):
    """Times PROBE["steps"] MP steps of the 384^3 x 4-species probe with CUDA events on the
    context's stream; returns the roofline entry of its step kernel (algorithmic bytes per
    step as for the main workload, per node-species)."""
    import torch
    from paper_1303_2470_gb300 import media
    n = PROBE["lattice"]
    solid, _ = media.random_spheres((n, n, n), PROBE["radius"], PROBE["porosity"], PROBE["seed"])
    u = torch.as_tensor(media.drift_flow(solid, 0.01, 0.01, seed=3).astype(np.float32)).cuda()
    Db, ka, kd = media.species(PROBE["species"], seed=PROBE["species_seed"], D_b=tuple(PROBE["D_b"]),
                               k=tuple(PROBE["k"]))
    stream = torch.cuda.Stream()
    steps = PROBE["steps"]
    ctx = mp.mp_init_batch(torch.as_tensor(solid).cuda(), u, Db, ka, kd, capacity=steps + 60, stream=stream,
                           **scheme_opts)
    del u
    mp.mp_step(ctx, 10)
    info = mp.mp_info(ctx)
    variant = mp.mp_variant(ctx)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    mp.mp_step(ctx, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    step_s = e0.elapsed_time(e1) / 1e3 / steps
    S, nf, ni = PROBE["species"], int(info["n_fluid"]), int(info["n_interface"])
    nbytes = nf * (16 * S + 13) + ni * 16 * S
    ctx.close()
    if variant == "flux":
        name, src = "k_step<float,multi>", "mp.cu"
    else:
        name = "k_direct_persistent" if variant.startswith("persistent") else "k_direct_step"
        src = "mp_direct.cu"
    tr = TRAFFIC.get(name + "@probe")
    traffic = tr["bytes_per_launch"] if tr and tr["src_sha"] == _src_sha(src) else None
    gbs = nbytes / step_s / 1e9
    return {"kernel": name, "variant": variant, "bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
            "frac": gbs / peak, "traffic": traffic, "algorithmic_bytes_per_step": nbytes,
            "us_per_step": step_s * 1e6, "node_species_updates_per_s": nf * S / step_s,
            "workload": f"random spheres {n}^3 (R={PROBE['radius']}, porosity {PROBE['porosity']}, seed "
                        f"{PROBE['seed']}), {S} species, {PROBE['flow']}; {nf} fluid, {ni} interfacial nodes; "
                        f"working set > 4x L2",
            "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
            else "fallback 6.8 TB/s"}


def mp_kernel_launches(variant, steps, tuned):
    """Kernels of mp_step(steps) and of the direct scheme's set-up: the flux scheme launches one
    kernel per step; the direct scheme one per step plus one that appends the last step's
    series per run (graphs of 64 steps are runs), or one persistent launch; its set-up adds
    the table kernel and, when tuned, 20 + 2 steps of each of the six one-step candidates (with
    their closing launches) and two launches of each of the six persistent ones."""
    if variant == "flux":
        return steps
    run = 1 if variant.startswith("persistent") else steps + -(-steps // 64)
    return run + 1 + (6 * (22 + 2) + 6 * 2 if tuned else 0)


def make_medium():
    from paper_1303_2470_gb300 import media
    nz, ny, nx = WORKLOAD["lattice"][::-1]
    solid, nspheres = media.random_spheres((nz, ny, nx), WORKLOAD["radius"], WORKLOAD["porosity"],
                                           WORKLOAD["seed"])
    return solid, nspheres


# ----------------------------------------------------------------------------------------
# oracle sample (CPU baseline and the reference arm)
# ----------------------------------------------------------------------------------------
def oracle_sample(solid, lb_steps_job, lb_sample=5, mp_sample=15):
    """Times the FP64 oracle as it stands on a bounded sample of the workload and scales
    it to one job: LB per-step time x lb_steps_job + MP setup + per-step time x 2e4."""
    import oracle
    oracle.build()
    F = (1e-5, 0.0, 0.0)
    f = oracle.lb_init(solid)
    t0 = time.perf_counter()
    for _ in range(lb_sample):
        f, u = oracle.lb_step(solid, f, F, WORKLOAD["tau"])
    t_lb = (time.perf_counter() - t0) / lb_sample
    p = oracle.Problem(solid, u, WORKLOAD["D_b"], WORKLOAD["k_a"], WORKLOAD["k_d"])
    t0 = time.perf_counter()
    oracle.run(p, g=0, nsteps=0)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.run(p, g=0, nsteps=mp_sample)
    t_mp = max(time.perf_counter() - t0 - t_setup, 1e-9) / mp_sample
    n_fluid = int((solid == 0).sum())
    job_s = t_lb * lb_steps_job + t_setup + t_mp * WORKLOAD["mp_steps"]
    value = n_fluid * WORKLOAD["species"] * WORKLOAD["mp_steps"] / job_s
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"oracle (FP64 C, OpenMP) on the same 128^3 medium: {lb_sample} LB steps "
              f"({t_lb*1e3:.0f} ms/step) and {mp_sample} MP steps ({t_mp*1e3:.0f} ms/step, setup "
              f"{t_setup:.1f} s), scaled to {lb_steps_job} LB steps + {WORKLOAD['mp_steps']} MP steps")
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "job_s_estimate": job_s}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    solid, _ = make_medium()
    for _ in range(args.warmup):
        oracle_sample(solid, LB_STEPS_ASSUMED, lb_sample=2, mp_sample=3)
    vals, wall = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        vals.append(oracle_sample(solid, LB_STEPS_ASSUMED))
        wall.append(time.perf_counter() - t0)
    value = statistics.median(v["value"] for v in vals)
    job_ms = statistics.median(v["job_s_estimate"] for v in vals) * 1e3
    cfg = dict(WORKLOAD)
    cfg["l2"] = "n/a (host)"
    # a step is one bounded sample (its wall time is ms_per_step); value is the sample's
    # rates scaled to the whole job, whose estimated duration is job_ms_estimate
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.median(wall) * 1e3,
            "job_ms_estimate": job_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {k: vals[-1][k] for k in ("kind", "cores", "sample")} | {"value": value,
                                                                                    "unit": UNIT},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------------------
BATCHED = {
    "workload": "three random-sphere media 64^3, 128^3, 192^3 (porosity U[0.35,0.5], radius "
                "U{4..8}, seeds 2-4), 16 species each (D_b U[0.01,0.1], k_a, k_d logU[1e-4,1e-1])",
    "sizes": [64, 128, 192],
    "seeds": [2, 3, 4],
    "species": 16,
    "mean_u": 0.01,
}


def run_batched(args):
    """Config of batched species and uneven media: every medium gets its LB flow, then all
    48 species advance (a) as one group of the three contexts, for each scheme (direct: the
    autotuned variant, one launch per step or one persistent launch; flux: one launch per
    step, CUDA graph, autotuned block), and (b) one species per launch (flux); all timed over
    the same number of steps. Grouped and one-species fields are identical for a scheme
    (tests/test_gpu_group.py, tests/test_gpu_direct.py), and both schemes meet the oracle bar
    on these media (tests/test_gpu_configs.py)."""
    import torch
    from paper_1303_2470_gb300 import build, media
    build.build()
    from paper_1303_2470_gb300 import mp
    rng = np.random.default_rng(2024)
    steps = max(args.mp_steps // 20, 200) if args.mp_steps else 500
    meds = []
    for n, seed in zip(BATCHED["sizes"], BATCHED["seeds"]):
        phi = float(rng.uniform(0.35, 0.5))
        solid, _ = media.random_spheres((n, n, n), [4, 5, 6, 7, 8], phi, seed)
        sd = torch.as_tensor(solid).cuda()
        u = torch.zeros((3,) + solid.shape, dtype=torch.float32, device="cuda")
        mp.lb_steady(sd, (1e-5, 0, 0), u, tol=1e-7, max_steps=100_000, check_every=100)
        fl = sd == 0
        F = 1e-5 * BATCHED["mean_u"] / float(u[0][fl].double().mean())
        lb_steps, _, _ = mp.lb_steady(sd, (F, 0, 0), u, tol=1e-7, max_steps=100_000, check_every=100)
        Db, ka, kd = media.species(BATCHED["species"], seed=seed + 100)
        meds.append((sd, u, Db, ka, kd, int(fl.sum()), phi, lb_steps))
    units = sum(m[5] for m in meds) * BATCHED["species"] * steps
    cap = 2 * steps + 40

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    grouped = {}
    for scheme in ("direct", "flux"):
        ctxs = [mp.mp_init_batch(sd, u, Db, ka, kd, capacity=cap, allow_negative=True, scheme=scheme)
                for sd, u, Db, ka, kd, *_ in meds]
        g = mp.mp_group_create(ctxs, graph_steps=64, autotune=True)
        mp.mp_group_step(g, 10)
        t = timed(lambda: mp.mp_group_step(g, steps))
        grouped[scheme] = {"updates_per_s": units / t, "ms_per_step": t / steps * 1e3,
                           "variant": mp.mp_group_variant(g), "block": mp.mp_group_block_size(g)}
        g.close()
        for c in ctxs:
            c.close()
    t_group = units / grouped["direct"]["updates_per_s"]
    singles = [mp.mp_init(sd, u, Db[s], ka[s], kd[s], capacity=cap, allow_negative=True)
               for sd, u, Db, ka, kd, *_ in meds for s in range(BATCHED["species"])]
    for c in singles:
        mp.mp_step(c, 10)

    def one_by_one():
        for _ in range(steps):
            for c in singles:
                mp.mp_step(c, 1)
    t_single = timed(one_by_one)
    for c in singles:
        c.close()
    line = {"metric": "batched sorption-MP node-species updates/s", "workload": BATCHED["workload"],
            "steps": steps, "grouped": units / t_group, "grouped_by_scheme": grouped,
            "one_species_per_launch": units / t_single, "one_species_per_launch_scheme": "flux",
            "speedup": t_single / t_group, "graph_steps": 64,
            "media": [{"n": int(m[0].shape[0]), "porosity": m[6], "n_fluid": m[5], "lb_steps": m[7]} for m in meds],
            "unit": UNIT}
    print(json.dumps(line))
    return 0


def warm_start_case(mp, surrogate, model, media, label, n, R, phi, seed, check=10, force=None, d_steps=0):
    """One medium solved by lb_steady to residual 1e-7 from rest and from the surrogate's warm
    start: steps, wall times (the warm time includes the network's inference), the estimate's
    error and the distance between the two converged flows; with d_steps > 0 also the largest
    relative difference of D(t) of the benchmark's tracer over d_steps MP steps on either flow.
    force: the body force; None calibrates it (untimed) to the benchmark's mean velocity 0.01."""
    import torch
    solid, _ = media.random_spheres((n, n, n), R, phi, seed)
    sd = torch.as_tensor(solid).cuda()
    fl = sd == 0
    u_cold = torch.zeros((3, n, n, n), dtype=torch.float32, device="cuda")
    if force is None:
        # Stokes-linear rescaling of a calibration solve (not timed)
        mp.lb_steady(sd, (1e-5, 0.0, 0.0), u_cold, tol=1e-7, max_steps=200_000, check_every=100)
        force = (1e-5 * WORKLOAD["mean_u"] / float(u_cold[0][fl].double().mean()), 0.0, 0.0)
        u_cold.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n_cold, _, c_cold = mp.lb_steady(sd, force, u_cold, tol=1e-7, max_steps=200_000, check_every=check)
    torch.cuda.synchronize()
    t_cold = time.perf_counter() - t0
    t0 = time.perf_counter()
    u0, rho0 = surrogate.warm_start(solid, force, model)
    torch.cuda.synchronize()
    t_inf = time.perf_counter() - t0
    u_warm = torch.zeros_like(u_cold)
    n_warm, _, c_warm = mp.lb_steady(sd, force, u_warm, tol=1e-7, max_steps=200_000, check_every=check,
                                     u_init=u0, rho_init=rho0)
    torch.cuda.synchronize()
    t_warm = time.perf_counter() - t0
    rec = {"case": label, "n": n, "radius": R, "porosity": round(phi, 4), "seed": seed, "force_x": force[0],
           "check_every": check, "cold_steps": int(n_cold), "warm_steps": int(n_warm),
           "converged": bool(c_cold and c_warm),
           "cold_s": round(t_cold, 4), "warm_s": round(t_warm, 4), "inference_s": round(t_inf, 4),
           "estimate_rel_l2": float((u0 - u_cold).norm() / u_cold.norm()),
           "flow_max_rel_diff": float((u_warm - u_cold).abs().max() / u_cold.abs().max())}
    if d_steps > 0:
        # the downstream observable: D(t) of the benchmark's tracer on either flow
        Ds = []
        for u in (u_cold, u_warm):
            ctx = mp.mp_init(sd, u, WORKLOAD["D_b"], WORKLOAD["k_a"], WORKLOAD["k_d"], capacity=d_steps + 2,
                             allow_negative=True)
            mp.mp_step(ctx, d_steps)
            Ds.append(mp.mp_vacf(ctx, 0, 0)[1])
            ctx.close()
        rec["D_steps"] = d_steps
        rec["D_max_rel_diff"] = float(np.max(np.abs(Ds[1] / Ds[0] - 1.0)))
    return rec


def forward_roofline(surrogate, model, n=128):
    """Tensor throughput of the network's forward pass on an n^3 box (all convolutions are
    3x3x3: 2 * 27 * Cin * Cout FLOPs per voxel and layer), CUDA events over five passes."""
    import torch
    x0 = torch.zeros((1, n ** 3, 16), dtype=torch.bfloat16, device="cuda")
    levels = {"e0a": 0, "e0b": 0, "e1a": 1, "e1b": 1, "e2a": 2, "e2b": 2, "b0": 3, "b1": 3, "d2a": 2, "d2b": 2,
              "d1a": 1, "d1b": 1, "d0a": 0, "d0b": 0, "out": 0}
    flops = sum(2.0 * 27 * cin * cout * (n >> levels[name]) ** 3 for name, cin, cout, _ in surrogate.LAYERS)
    model.forward(x0, 1, (n, n, n))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(5):
        model.forward(x0, 1, (n, n, n))
    e1.record()
    torch.cuda.synchronize()
    fwd_s = e0.elapsed_time(e1) / 5e3
    peak = None
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pp):
        peak = json.load(open(pp)).get("bf16_tflops")
    return {"kernel": f"k_conv_row + k_conv_tc (forward pass, {n}^3 box)", "bound": "tensor",
            "achieved": flops / fwd_s / 1e12,
            "peak": peak, "unit": "TFLOP/s", "frac": (flops / fwd_s / 1e12 / peak) if peak else None,
            "flops": flops, "ms": fwd_s * 1e3,
            "peak_source": "measured (MEASURED_PEAKS.json bf16_tflops, burst)" if peak else "unavailable"}


def run_warm_start_record(mp, force_x):
    """The default line's record of the learned warm start: an unseen 256^3 medium (spheres
    R = 6, porosity 0.40, seed 90101) from rest and from the warm start at the benchmark's
    force, with D(t) over 1000 MP steps on either flow, and the forward pass's tensor
    throughput on a 128^3 box."""
    from paper_1303_2470_gb300 import media, surrogate
    model, meta = surrogate.load()
    rec = warm_start_case(mp, surrogate, model, media, "unseen 256^3", 256, 6, 0.40, 90_101,
                          force=(force_x, 0.0, 0.0), d_steps=1000)
    return {"steps_factor": rec["cold_steps"] / rec["warm_steps"], "time_factor": rec["cold_s"] / rec["warm_s"],
            "case": rec, "tensor_roofline": forward_roofline(surrogate, model),
            "model": {"n_params": meta["n_params"], "train_media": meta["n_train"], "size": meta["size"]}}


def run_surrogate(args):
    """LB warm start from the trained surrogate against the cold start (both to residual
    1e-7, checked every 10 steps, at the force giving the benchmark's mean interstitial
    velocity 0.01): unseen 64^3 media, the benchmark's 128^3 medium and unseen 256^3 media. Reports steps and wall time (the warm time includes the network's inference),
    the estimate's error, the distance between the two converged flows and, on the benchmark
    medium, the largest relative difference of D(t) over 2000 MP steps run on either flow."""
    import torch
    from paper_1303_2470_gb300 import build, media
    build.build()
    from paper_1303_2470_gb300 import mp, surrogate
    model, meta = surrogate.load()
    rng = np.random.default_rng(77)
    cases = [("unseen 64^3", 64, int(rng.integers(4, 9)), float(rng.uniform(0.3, 0.6)), 90_001 + i) for i in range(8)]
    cases += [("benchmark medium 128^3", 128, WORKLOAD["radius"], WORKLOAD["porosity"], WORKLOAD["seed"])]
    cases += [("unseen 256^3", 256, 6, 0.40, 90_101), ("unseen 256^3", 256, 5, 0.50, 90_102)]
    out = []
    for label, n, R, phi, seed in cases:
        rec = warm_start_case(mp, surrogate, model, media, label, n, R, phi, seed,
                              d_steps=2000 if label.startswith("benchmark") else 0)
        out.append(rec)
        print(json.dumps(rec), flush=True)
    tensor = forward_roofline(surrogate, model)
    line = {"metric": "LB steps to residual 1e-7: cold start / surrogate warm start", "unit": "ratio",
            "steps_factor": {c: float(np.mean([r["cold_steps"] / r["warm_steps"] for r in out if r["case"] == c]))
                             for c in dict.fromkeys(r["case"] for r in out)},
            "time_factor": {c: float(np.mean([r["cold_s"] / r["warm_s"] for r in out if r["case"] == c]))
                            for c in dict.fromkeys(r["case"] for r in out)},
            "cases": out,
            "tensor_roofline": tensor,
            "model": {"n_params": meta["n_params"], "train_media": meta["n_train"], "size": meta["size"],
                      "iters": meta["iters"], "batch": meta["batch"], "train_seconds": meta["train_seconds"],
                      "final_loss": meta["loss_history"][-1][1]}}
    print(json.dumps(line))
    return 0


def run_profile_probe(args):
    """A smaller case of the beyond-L2 probe for ncu --set full captures (python bench.py
    --profile-probe): 192^3 random spheres (R = 6, porosity 0.40, seed 1) x 4 species, about
    1 GB on the device, 20 MP steps with the scheme and variant given."""
    import torch
    from paper_1303_2470_gb300 import build, media
    build.build()
    from paper_1303_2470_gb300 import mp
    n = 192
    solid, _ = media.random_spheres((n, n, n), PROBE["radius"], PROBE["porosity"], PROBE["seed"])
    u = torch.as_tensor(media.drift_flow(solid, 0.01, 0.01, seed=3).astype(np.float32)).cuda()
    Db, ka, kd = media.species(PROBE["species"], seed=PROBE["species_seed"], D_b=tuple(PROBE["D_b"]),
                               k=tuple(PROBE["k"]))
    ctx = mp.mp_init_batch(torch.as_tensor(solid).cuda(), u, Db, ka, kd, capacity=64, **scheme_options(args))
    mp.mp_step(ctx, 20)
    torch.cuda.synchronize()
    info = mp.mp_info(ctx)
    print(json.dumps({"profile_probe": "ok", "n_fluid": info["n_fluid"], "n_interface": info["n_interface"],
                      "variant": mp.mp_variant(ctx)}))
    ctx.close()
    return 0


def run_profile_batched(args):
    """Two random-sphere media (96^3, 128^3) x 16 species, 30 LB steps each, then 8 grouped
    steps without graph or autotune, in the scheme and variant given: `k_step_group` (flux)
    or `k_direct_step` / `k_direct_persistent` (direct) launches for ncu captures."""
    import torch
    from paper_1303_2470_gb300 import build, media
    build.build()
    from paper_1303_2470_gb300 import mp
    ctxs = []
    for n, seed in ((96, 2), (128, 3)):
        solid, _ = media.random_spheres((n, n, n), [4, 5, 6, 7, 8], 0.42, seed)
        sd = torch.as_tensor(solid).cuda()
        u = torch.zeros((3,) + solid.shape, dtype=torch.float32, device="cuda")
        mp.lb_steady(sd, (1e-3, 0, 0), u, tol=0.0, max_steps=30, check_every=30)
        Db, ka, kd = media.species(16, seed=seed + 100)
        opts = scheme_options(args)
        opts.pop("autotune", None)
        variant = opts.pop("variant", 0)
        ctxs.append(mp.mp_init_batch(sd, u, Db, ka, kd, capacity=16, allow_negative=True, **opts))
    g = mp.mp_group_create(ctxs, variant=variant)
    mp.mp_group_step(g, 8)
    torch.cuda.synchronize()
    print(json.dumps({"profile_batched": "ok", "block": mp.mp_group_block_size(g), "variant": mp.mp_group_variant(g)}))
    g.close()
    return 0


def run_profile_surrogate():
    """Two forward passes of the trained warm-start network on a 128^3 box, no timing: for ncu
    captures of the tensor-core convolutions. Per pass, in layer order, the five layers at full
    resolution (e0a, e0b, d0a, d0b, out) run `k_conv_row` and the ten coarser ones `k_conv_tc`;
    the second pass's d0a (64 -> 32 channels) is `k_conv_row` launch 7."""
    import torch
    from paper_1303_2470_gb300 import build
    build.build()
    from paper_1303_2470_gb300 import surrogate
    model, _ = surrogate.load()
    n = 128
    x0 = torch.zeros((1, n ** 3, 16), dtype=torch.bfloat16, device="cuda")
    for _ in range(2):
        model.forward(x0, 1, (n, n, n))
    torch.cuda.synchronize()
    print(json.dumps({"profile_surrogate": "ok", "layers": [name for name, _, _, _ in surrogate.LAYERS]}))
    return 0


def scheme_options(args):
    """mp_init options of the MP step's evaluation: the scheme, and for the direct scheme
    the autotuner or a fixed kernel variant."""
    if args.scheme == "flux" or args.precision == "fp16":
        return {"scheme": "flux"}
    return {"scheme": "direct", "autotune": args.variant < 0, "variant": max(args.variant, 0)}


def run_profile_case(args):
    """The workload's kernels on the same 128^3 medium, briefly, for ncu --set full
    captures (python bench.py --profile): LB launches 1-30, k_init, MP launches 1-20."""
    import torch
    from paper_1303_2470_gb300 import build
    build.build()
    from paper_1303_2470_gb300 import mp
    solid, _ = make_medium()
    sd = torch.as_tensor(solid).cuda()
    u = torch.zeros((3,) + solid.shape, dtype=torch.float32, device="cuda")
    mp.lb_steady(sd, (1.83e-3, 0, 0), u, tau=WORKLOAD["tau"], tol=0.0, max_steps=30, check_every=30)
    ctx = mp.mp_init(sd, u, WORKLOAD["D_b"], WORKLOAD["k_a"], WORKLOAD["k_d"], allow_negative=True, capacity=64,
                     **scheme_options(args))
    mp.mp_step(ctx, 20)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": "ok", "n_fluid": mp.mp_info(ctx)["n_fluid"], "variant": mp.mp_variant(ctx)}))
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-warm-start", action="store_true",
                    help="leave out the learned warm start's record (an unseen 256^3 medium) of the default line")
    ap.add_argument("--no-probe", action="store_true",
                    help="skip the 384^3 x 4-species probe of the step beyond L2 (roofline_hbm)")
    ap.add_argument("--mp-steps", type=int, default=WORKLOAD["mp_steps"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16"],
                    help="field storage of the MP step: fp32 (default) or binary16 with FP32 "
                         "arithmetic and stochastic rounding")
    ap.add_argument("--workload", default="porous128", choices=["porous128", "batched", "surrogate"],
                    help="porous128: the single-species 128^3 job (the bench line); batched: three "
                         "media x 16 species, grouped launch vs one species per launch; surrogate: LB "
                         "steps to steady from the learned warm start vs the cold start")
    ap.add_argument("--profile-batched", action="store_true",
                    help="short grouped run (96^3 and 128^3 media x 16 species) for ncu captures")
    ap.add_argument("--profile-probe", action="store_true",
                    help="20 MP steps of a 192^3 x 4-species case of the beyond-L2 probe for ncu captures")
    ap.add_argument("--profile-surrogate", action="store_true",
                    help="two forward passes of the warm-start network on a 128^3 box for ncu captures")
    ap.add_argument("--scheme", default="direct", choices=["direct", "flux"],
                    help="evaluation of the MP step: direct (the paper's form with per-node link "
                         "tables, default) or flux (exactly antisymmetric link fluxes)")
    ap.add_argument("--variant", type=int, default=-1,
                    help="direct scheme: MP_VARIANT_* flags of a fixed kernel variant, or -1 (default) "
                         "to let mp_init autotune it")
    ap.add_argument("--profile", action="store_true",
                    help="short run of the same medium and kernels for ncu captures: 30 LB steps, "
                         "mp_init and 20 MP steps, no timing")
    args = ap.parse_args()
    WORKLOAD["mp_steps"] = args.mp_steps
    if args.impl == "reference":
        return run_reference(args)
    if args.profile:
        return run_profile_case(args)
    if args.profile_batched:
        return run_profile_batched(args)
    if args.profile_probe:
        return run_profile_probe(args)
    if args.profile_surrogate:
        return run_profile_surrogate()
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "surrogate":
        return run_surrogate(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_1303_2470_gb300 import build
    build.build()
    from paper_1303_2470_gb300 import mp

    solid, nspheres = make_medium()
    n_fluid = int((solid == 0).sum())
    solid_dev = torch.as_tensor(solid).to(dev)
    stream = torch.cuda.current_stream(dev)
    u = torch.zeros((3,) + solid.shape, dtype=torch.float32, device=dev)

    # force set once (Stokes-linear): mean fluid u_x = 0.01
    F0 = 1e-5
    mp.lb_steady(solid_dev, (F0, 0, 0), u, tau=WORKLOAD["tau"], tol=WORKLOAD["lb_tol"],
                 max_steps=200_000, check_every=WORKLOAD["lb_check_every"], stream=stream)
    mean0 = float(u[0][solid_dev == 0].double().mean())
    Fx = F0 * WORKLOAD["mean_u"] / mean0
    force = (Fx, 0.0, 0.0)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2

    def job(solid_arg, host_out=None):
        """One pass of the whole path. Returns (lb_steps, ctx info, event list)."""
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        steps, res, conv = mp.lb_steady(solid_arg, force, u, tau=WORKLOAD["tau"], tol=WORKLOAD["lb_tol"],
                                        max_steps=200_000, check_every=WORKLOAD["lb_check_every"],
                                        stream=stream)
        ev[1].record(stream)
        ctx = mp.mp_init(solid_arg, u, WORKLOAD["D_b"], WORKLOAD["k_a"], WORKLOAD["k_d"],
                         capacity=WORKLOAD["mp_steps"] + 26, stream=stream, allow_negative=True,
                         precision=args.precision, **scheme_options(args))
        ev[2].record(stream)
        mp.mp_step(ctx, WORKLOAD["mp_steps"])
        if host_out is not None:
            mp.mp_vacf_into(ctx, 0, 0, host_out[0], host_out[1])
        ev[3].record(stream)
        info = mp.mp_info(ctx)
        info["variant"] = mp.mp_variant(ctx)
        return steps, res, conv, info, ev, ctx

    for _ in range(args.warmup):
        *_, ctx = job(solid_dev)
        torch.cuda.synchronize()
        ctx.close()

    clocks = ClockSampler(dev.index)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    total_ms, lb_ms, init_ms, mp_ms, lb_steps_all, launches = 0.0, 0.0, 0.0, 0.0, [], 0
    info = None
    for _ in range(args.steps):
        flush.fill_(1.0)  # evict the previous job's data from L2 (outside the timed events)
        steps, res, conv, info, ev, ctx = job(solid_dev)
        torch.cuda.synchronize()
        total_ms += ev[0].elapsed_time(ev[3])
        lb_ms += ev[0].elapsed_time(ev[1])
        init_ms += ev[1].elapsed_time(ev[2])
        mp_ms += ev[2].elapsed_time(ev[3])
        lb_steps_all.append(steps)
        # kernels: the LB and MP steps, one two-iterate mean per failed residual check, and
        # the job's one-off kernels (geometry, cluster labelling, initialisation)
        launches += (steps + max(steps // WORKLOAD["lb_check_every"] - 1, 0) + JOB_FIXED_LAUNCHES
                     + mp_kernel_launches(info["variant"], WORKLOAD["mp_steps"], args.variant < 0))
        ctx.close()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    units_per_job = n_fluid * WORKLOAD["species"] * WORKLOAD["mp_steps"]
    slowest_s, value = aggregate(total_ms / 1e3, units_per_job * args.steps, world, dist, dev)
    total_ms_max = slowest_s * 1e3

    # end to end through the public API: host solid mask in, host Z(t)/D(t) out
    Zh = torch.empty(WORKLOAD["mp_steps"] + 2, dtype=torch.float64, pin_memory=True).numpy()
    Dh = torch.empty(WORKLOAD["mp_steps"] + 2, dtype=torch.float64, pin_memory=True).numpy()
    e2e_s = 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        *_, ctx = job(solid, host_out=(Zh, Dh))
        torch.cuda.synchronize()
        e2e_s += time.perf_counter() - t0
        ctx.close()
    _, e2e_value = aggregate(e2e_s, units_per_job * args.steps, world, dist, dev)

    # roofline of the dominant kernel, from the live event timings above
    peak, peak_kind = _peaks()
    n_iface = int(info["n_interface"])
    S = WORKLOAD["species"]
    eb = 2 if args.precision == "fp16" else 4                     # bytes per stored field value
    variant = info["variant"]
    if variant == "flux":
        mp_name, mp_src = ("k_step<float,half>" if args.precision == "fp16" else "k_step<float>"), "mp.cu"
    else:
        # a persistent launch runs the whole run of steps: its per-step time is the unit
        mp_name = "k_direct_persistent" if variant.startswith("persistent") else "k_direct_step"
        mp_src = "mp_direct.cu"
    # per MP launch: 2 fields read + written per fluid node and species, flow 12 B + flags 1 B
    # per fluid node, the adsorbed partners' 2 fields read + written per interfacial node
    mp_bytes = n_fluid * (4 * eb * S + 13) + n_iface * 4 * eb * S
    lb_steps_mean = float(np.mean(lb_steps_all))
    lb_bytes = n_fluid * 19 * 2 * 4                               # per LB launch
    mp_launch_s = mp_ms / 1e3 / (args.steps * WORKLOAD["mp_steps"])
    lb_launch_s = lb_ms / 1e3 / (args.steps * lb_steps_mean)
    kern = {
        mp_name: {"share": mp_ms / total_ms, "avg_launch_us": mp_launch_s * 1e6,
                          "algorithmic_bytes": mp_bytes, "gbs": mp_bytes / mp_launch_s / 1e9,
                          "src": mp_src, "variant": variant},
        "k_lb_step": {"share": lb_ms / total_ms, "avg_launch_us": lb_launch_s * 1e6,
                      "algorithmic_bytes": lb_bytes, "gbs": lb_bytes / lb_launch_s / 1e9, "src": "lb.cu"},
    }
    dom = max(kern, key=lambda k: kern[k]["share"])
    tr = TRAFFIC.get(dom)
    traffic = tr["bytes_per_launch"] if tr and tr["src_sha"] == _src_sha(kern[dom]["src"]) else None
    roofline = {"kernel": dom, "bound": "hbm", "achieved": kern[dom]["gbs"], "peak": peak, "unit": "GB/s",
                "frac": kern[dom]["gbs"] / peak, "traffic": traffic,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                else "fallback 6.8 TB/s"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(WORKLOAD, n_fluid=n_fluid, n_interface=n_iface, spheres=nspheres,
                       **({"precision": "binary16 field storage (stochastic rounding), fp32 arithmetic, "
                                        "fp64 reductions and D(t)"} if args.precision == "fp16" else {}),
                       negative_links=int(info["n_negative_links"]),
                       force_x=Fx, l2="256 MiB buffer written between timed jobs",
                       parallelism="replicas" if world > 1 else "single GPU"),
        "lb": {"steps_to_steady": lb_steps_all, "ms": lb_ms / args.steps,
               "mlups": n_fluid * lb_steps_mean / (lb_ms / args.steps / 1e3) / 1e6,
               "check_every": WORKLOAD["lb_check_every"], "tol": WORKLOAD["lb_tol"],
               "iteration": "BGK steps; at every failed residual check the populations are replaced by the "
                            "mean of the last two iterates (reading R16), so steps_to_steady counts steps "
                            "of that iteration"},
        "mp": {"ms": mp_ms / args.steps, "init_ms": init_ms / args.steps,
               "kernel_rate": units_per_job / (mp_ms / args.steps / 1e3)},
        "kernels": kern,
        "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * int(solid.size),
                "d2h_bytes_per_step": 2 * 8 * (WORKLOAD["mp_steps"] + 2)},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if rank == 0 and not args.no_probe:
        line["roofline_hbm"] = run_hbm_probe(mp, peak, peak_kind, scheme_options(args))
    if rank == 0 and not args.no_warm_start:
        line["warm_start"] = run_warm_start_record(mp, Fx)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample(solid, int(round(lb_steps_mean)))
        line["cpu_baseline"].pop("job_s_estimate", None)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
