"""The paper's validation experiments (Sec. Validation), run through the library.

Each function sets up one of the paper's synthetic systems, advances it on the GPU through
the C ABI and returns the raw series; comparisons with exact solutions are left to the
caller. Media and flows come from `media`; nothing here computes a propagation step.

  * slit_wall_normal -- Figs. 1 and 2: D(t) normal to the walls of a slit pore of width L
    for several sorption pairs (k_a, k_d), one species per pair in one batched context;
  * taylor_aris      -- Fig. 3: D(t) along a Poiseuille flow in the slit, one context per
    Peclet number Pe = L vbar/D_b (vbar the mean fluid velocity), species = sorption pairs;
  * fcc_packing      -- Fig. 5: D(t) in a periodic fcc unit cell of touching spheres for
    several adsorbed fractions f_a, one species per f_a.
"""
from __future__ import annotations

import numpy as np

from . import media
from . import mp


def _series(ctx, n_species, direction, times):
    times = np.asarray(times, dtype=np.int64)
    Z = np.zeros((n_species, times.size))
    D = np.zeros((n_species, times.size))
    for s in range(n_species):
        z, d = mp.mp_vacf(ctx, s, direction, cap=int(times.max()) + 1)
        Z[s] = z[times]
        D[s] = d[times]
    return Z, D


def _run(ctxs, steps, chunk=1024):
    """Advance every context `steps` steps, alternating in short chunks (replayed from CUDA
    graphs) so that the contexts' launches, each on its own stream, overlap on the device."""
    done = 0
    while done < steps:
        n = min(chunk, steps - done)
        for c in ctxs:
            mp.mp_step(c, n)
        done += n


def slit_wall_normal(pairs, L=100, D_b=0.01, steps=1_000_000, times=None, precision="fp64", width=3,
                     species_per_context=1):
    """D_z(t) of a slit of L fluid planes (walls normal to z) for each (k_a, k_d) in pairs.
    The pairs are spread over contexts of up to species_per_context species, each on its
    own stream, so that the small lattice's launches run side by side on the device.
    Returns dict(times, Z[species, len(times)], D[...], mass[species, 3], n_interface)."""
    import torch

    pairs = [(float(a), float(d)) for a, d in pairs]
    times = np.arange(steps + 1) if times is None else np.asarray(times, dtype=np.int64)
    solid = media.slit(width, width, L)
    groups = [pairs[i:i + species_per_context] for i in range(0, len(pairs), species_per_context)]
    streams = [torch.cuda.Stream() for _ in groups]
    ctxs = []
    try:
        for grp, st in zip(groups, streams):
            ctxs.append(mp.mp_init_batch(solid, None, [D_b] * len(grp), [p[0] for p in grp], [p[1] for p in grp],
                                         precision=precision, directions="z", capacity=steps + 2, stream=st))
        _run(ctxs, steps)
        Z, D, mass = [], [], []
        for c, grp in zip(ctxs, groups):
            z, d = _series(c, len(grp), 2, times)
            Z.append(z)
            D.append(d)
            mass += [mp.mp_mass(c, s) for s in range(len(grp))]
        info = mp.mp_info(ctxs[0])
    finally:
        for c in ctxs:
            c.close()
    return {"times": times, "Z": np.concatenate(Z), "D": np.concatenate(D), "mass": np.array(mass),
            "n_interface": info["n_interface"]}


def poiseuille_u_max(L, D_b, Pe):
    """u_max of the slit's parabolic profile (media.poiseuille_profile) whose mean over the
    L fluid planes gives Pe = L vbar / D_b."""
    unit = media.poiseuille_profile(L, 1.0)[1:L + 1].mean()
    return Pe * D_b / (L * unit)


def taylor_aris(Pes, pairs, L=100, D_b=0.01, steps=1_000_000, times=None, precision="fp64", width=3,
                allow_negative=False):
    """D_x(t) along a Poiseuille flow for each Peclet number in Pes and each sorption pair,
    one single-species context per (Pe, pair), each on its own stream. The flow is passed
    to the library in FP32, as every flow is.
    Returns dict(times, u_max[len(Pes)], Z[pe, species, t], D[pe, species, t])."""
    import torch

    pairs = [(float(a), float(d)) for a, d in pairs]
    times = np.arange(steps + 1) if times is None else np.asarray(times, dtype=np.int64)
    solid = media.slit(width, width, L)
    ctxs, umaxs, streams = [], [], []
    try:
        for Pe in Pes:
            umax = poiseuille_u_max(L, D_b, Pe)
            umaxs.append(umax)
            u = torch.as_tensor(media.slit_flow(width, width, L, umax).astype(np.float32)).cuda()
            torch.cuda.synchronize()
            for ka, kd in pairs:
                streams.append(torch.cuda.Stream())
                ctxs.append(mp.mp_init(solid, u, D_b, ka, kd, precision=precision, directions="x",
                                       capacity=steps + 2, allow_negative=allow_negative, stream=streams[-1]))
            del u  # mp_init copied the flow and synchronised its stream
        _run(ctxs, steps)
        out = [_series(c, 1, 0, times) for c in ctxs]
    finally:
        for c in ctxs:
            c.close()
    shape = (len(Pes), len(pairs), times.size)
    return {"times": times, "u_max": np.array(umaxs), "Z": np.stack([o[0][0] for o in out]).reshape(shape),
            "D": np.stack([o[1][0] for o in out]).reshape(shape)}


def fcc_sorption_pairs(solid, fractions, k_a=0.1):
    """(k_a, k_d) giving each adsorbed fraction f_a at equilibrium on this medium:
    f_a = K n_I / (n_F + K n_I) with K = k_a/k_d (the Boltzmann weights of the method),
    n_F fluid and n_I interfacial nodes. f_a = 0 gives (0, 0)."""
    _, (nf, ni, _) = mp.mp_classify(solid)
    pairs = []
    for f in fractions:
        if f == 0.0:
            pairs.append((0.0, 0.0))
        else:
            K = f / (1.0 - f) * nf / ni
            pairs.append((k_a, k_a / K))
    return pairs


def fcc_packing(a=100, fractions=(0.0, 0.30, 0.79, 0.97), D_b=0.01, k_a=0.1, steps=None, reduced_time=2.0,
                times=None, precision="fp32"):
    """D_x(t) in one periodic fcc unit cell of lattice parameter a (touching spheres,
    R = a sqrt(2)/4) for each adsorbed fraction. steps defaults to reduced_time R^2/D_b.
    Returns dict(times, R, pairs, Z, D, mass, porosity)."""
    solid = media.fcc(a)
    R = a * np.sqrt(2.0) / 4.0
    if steps is None:
        steps = int(round(reduced_time * R * R / D_b))
    times = np.arange(steps + 1) if times is None else np.asarray(times, dtype=np.int64)
    pairs = fcc_sorption_pairs(solid, fractions, k_a)
    n = len(pairs)
    ctx = mp.mp_init_batch(solid, None, [D_b] * n, [p[0] for p in pairs], [p[1] for p in pairs],
                           precision=precision, directions="x", capacity=steps + 2)
    try:
        _run([ctx], steps)
        Z, D = _series(ctx, n, 0, times)
        mass = np.array([mp.mp_mass(ctx, s) for s in range(n)])
        info = mp.mp_info(ctx)
    finally:
        ctx.close()
    return {"times": times, "R": R, "pairs": pairs, "Z": Z, "D": D, "mass": mass,
            "porosity": info["n_fluid"] / info["n_nodes"], "n_fluid": info["n_fluid"],
            "n_interface": info["n_interface"]}
