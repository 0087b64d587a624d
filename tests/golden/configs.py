"""Stored oracle series of two full-size workloads, and the script that writes them.

The FP64 oracle needs about an hour of host time for the porous-medium workload below
(2e4 steps on 838,771 fluid nodes), too long for a test, so its Z(t) and D(t) are computed
once by this script and stored as JSON next to it. The script calls only the oracle
(``oracle/``) and the seeded input generators (``paper_1303_2470_gb300/media.py``); no value
comes from the CUDA library. The GPU tests rebuild the same inputs from the same seeds.

Workloads (inputs seeded and synthetic; the flow is a seeded drift plus noise, identical on
both sides, rounded to FP32 because the library takes FP32 velocities):
  porous128  -- random-sphere medium 128^3, radius 6, porosity 0.40, seed 1; one species
                D_b = 0.05, k_a = k_d = 5e-3; flow mean 0.01 along x, noise 0.01; 2e4 steps;
                x moment (paper Sec. "Algorithm": the velocity-weighted propagated quantity,
                Z(t) its VACF sum, D(t) = Z(0)/2 + sum Z).
  batched    -- three random-sphere media 64^3, 128^3, 192^3 (porosity U[0.35, 0.5] from
                generator seed 2024, radii U{4..8}, seeds 2, 3, 4), 16 species per medium
                (D_b U[0.01, 0.1], k_a, k_d logU[1e-4, 1e-1], seed 100 + medium seed); the
                oracle runs all 16 species of the 64^3 medium and species 0 and 1 of the
                two larger ones; flow mean 0.005 along x, noise 0.004 (all p_i > 0);
                1e3 steps; x moment.

Run ``python tests/golden/configs.py [porous128|batched]`` to rewrite the files.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1303_2470_gb300 import media  # noqa: E402  (seeded input generators only)

PATHS = {"porous128": os.path.join(HERE, "porous128_series.json"),
         "batched": os.path.join(HERE, "batched_series.json")}


def sample_times(T: int):
    """Stored time points of a series with entries t = 0..T: every step up to 200, then
    every 25 steps, and T."""
    ts = set(range(0, min(T, 200) + 1)) | set(range(200, T + 1, 25)) | {T}
    return sorted(t for t in ts if t <= T)


def porous128():
    """(solid, u32[3,...], D_b, k_a, k_d, nsteps) of the porous-medium workload."""
    solid, _ = media.random_spheres((128, 128, 128), 6, 0.40, seed=1)
    u = media.drift_flow(solid, 0.01, 0.01, seed=3).astype(np.float32)
    return solid, u, 0.05, 5e-3, 5e-3, 20_000


def batched():
    """List of media (solid, u32, (D_b, k_a, k_d) arrays of 16 species, oracle species
    indices) and the step count of the batched workload."""
    rng = np.random.default_rng(2024)
    out = []
    for n, seed in zip((64, 128, 192), (2, 3, 4)):
        phi = float(rng.uniform(0.35, 0.5))
        solid, _ = media.random_spheres((n, n, n), [4, 5, 6, 7, 8], phi, seed)
        u = media.drift_flow(solid, 0.005, 0.004, seed=seed + 200).astype(np.float32)
        sp = media.species(16, seed=seed + 100)
        checked = list(range(16)) if n == 64 else [0, 1]
        out.append((solid, u, sp, checked))
    return out, 1_000


def _series(run, T):
    ts = sample_times(T)
    return {"t": ts, "Z": [float(run.Z[t]) for t in ts], "D": [float(run.D[t]) for t in ts],
            "mass_free": float(run.mass_free[T]), "mass_ads": float(run.mass_ads[T])}


def write_porous128():
    import oracle
    solid, u, Db, ka, kd, steps = porous128()
    t0 = time.time()
    r = oracle.run(oracle.Problem(solid, u.astype(np.float64), Db, ka, kd), g=0, nsteps=steps)
    rec = {"workload": "porous128", "steps": steps, "direction": 0, "n_fluid": int((solid == 0).sum()),
           "series": [_series(r, steps + 1)], "oracle_seconds": round(time.time() - t0, 1)}
    with open(PATHS["porous128"], "w") as f:
        json.dump(rec, f)


def write_batched():
    import oracle
    meds, steps = batched()
    series = []
    t0 = time.time()
    for m, (solid, u, (Db, ka, kd), checked) in enumerate(meds):
        u64 = u.astype(np.float64)
        for s in checked:
            r = oracle.run(oracle.Problem(solid, u64, Db[s], ka[s], kd[s]), g=0, nsteps=steps)
            series.append({"medium": m, "species": s} | _series(r, steps + 1))
    rec = {"workload": "batched", "steps": steps, "direction": 0, "series": series,
           "oracle_seconds": round(time.time() - t0, 1)}
    with open(PATHS["batched"], "w") as f:
        json.dump(rec, f)


if __name__ == "__main__":
    which = sys.argv[1:] or ["porous128", "batched"]
    for w in which:
        {"porous128": write_porous128, "batched": write_batched}[w]()
        print("wrote", PATHS[w])
