"""Split of independent moment-propagation problems over the ranks of a job.

Species in a medium, and media, are independent problems: the step of one never reads the
fields of another (paper Sec. "Algorithm": each tracer species propagates on its own, with its
own D_b, k_a, k_d, over the shared steady flow). A multi-GPU job therefore needs no exchange
while it steps. The units (medium, species) are dealt to the ranks in balanced contiguous
runs; every rank advances its units with the library (one context per medium holding that
rank's species of it) and, once at the end, the Z(t) and D(t) series of all units are
gathered to every rank. This module only assigns units, marshals calls to the C ABI and
gathers the series; it does none of the method's arithmetic.
"""
from __future__ import annotations

import numpy as np


def split_units(units, world):
    """Balanced contiguous runs of `units` for ranks 0..world-1: rank r gets
    units[floor(r n / world) : floor((r+1) n / world)]."""
    n = len(units)
    return [list(units[(r * n) // world:((r + 1) * n) // world]) for r in range(world)]


def gather_series(local, dist=None, world=1):
    """Merges the per-rank dictionaries {unit: (Z, D)} into one dictionary held by every
    rank (all-gather of Python objects; a single rank returns its own). Units must be
    distinct across ranks."""
    if world == 1 or dist is None:
        return dict(local)
    parts = [None] * world
    dist.all_gather_object(parts, {k: (np.asarray(z), np.asarray(d)) for k, (z, d) in local.items()})
    merged = {}
    for p in parts:
        for k, v in p.items():
            if k in merged:
                raise ValueError(f"unit {k} was run by two ranks")
            merged[k] = v
    return merged


def run_units(media, units, steps, run_medium):
    """Runs `units` (pairs (medium index, species index)) for `steps` steps: for every medium
    that has units, run_medium(medium, species_indices, steps) returns {species: (Z, D)}.
    Returns {(medium, species): (Z, D)}."""
    by_medium = {}
    for m, s in units:
        by_medium.setdefault(m, []).append(s)
    out = {}
    for m, species in sorted(by_medium.items()):
        res = run_medium(media[m], species, steps)
        for s in species:
            out[(m, s)] = res[s]
    return out


def mp_medium_runner(mp, direction=0, **options):
    """run_medium for run_units through the library: media[m] = (solid, u, (D_b, k_a, k_d))
    with u a device FP32 buffer (or None); one context with the requested species."""
    def run(medium, species, steps):
        solid, u, (Db, ka, kd) = medium
        idx = list(species)
        ctx = mp.mp_init_batch(solid, u, np.asarray(Db)[idx], np.asarray(ka)[idx], np.asarray(kd)[idx],
                               capacity=steps + 30, **options)
        try:
            mp.mp_step(ctx, steps)
            return {s: mp.mp_vacf(ctx, j, direction) for j, s in enumerate(idx)}
        finally:
            ctx.close()
    return run


def run_sharded(media, units, steps, run_medium, rank=0, world=1, dist=None):
    """The whole split: this rank's share of `units`, run, then the gather. Every rank
    returns the series of all units."""
    mine = split_units(units, world)[rank]
    return gather_series(run_units(media, mine, steps, run_medium), dist, world)
