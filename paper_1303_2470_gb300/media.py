"""Seeded synthetic inputs: solid masks, flow fields and tracer species.

This module holds none of the moment-propagation arithmetic; it only makes the inputs
that both the GPU library and the FP64 oracle are fed. All arrays use the lattice layout
of the library: shape (nz, ny, nx), x fastest, periodic on every axis, solid = 1.

Geometries follow the media of the paper: the slit pore of its validation section, the
compact face-centred cubic packing of spheres of its porous-medium example, and, for the
large porous-medium workloads, randomly placed overlapping spheres (a Boolean model).
"""
from __future__ import annotations

import numpy as np


def slit(nx: int, ny: int, H: int) -> np.ndarray:
    """Slit pore: H fluid planes between two solid planes, z = 0 and z = H+1.
    Returns solid[H+2, ny, nx] (uint8)."""
    s = np.zeros((H + 2, ny, nx), dtype=np.uint8)
    s[0] = 1
    s[H + 1] = 1
    return s


def bulk(nx: int, ny: int, nz: int) -> np.ndarray:
    """Periodic box with no solid."""
    return np.zeros((nz, ny, nx), dtype=np.uint8)


def fcc(a: int, radius: float | None = None) -> np.ndarray:
    """One periodic unit cell of a face-centred cubic packing of spheres (Sec. Validation,
    the fcc example): lattice parameter a nodes, sphere centres at the cell corner and the
    three face centres, (0,0,0), (a/2,a/2,0), (a/2,0,a/2), (0,a/2,a/2), with their periodic
    images. radius defaults to the compact (touching) packing, a sqrt(2)/4, whose continuum
    porosity is 1 - pi/(3 sqrt 2) ~ 0.26. Node (x,y,z) sits at integer coordinates and is
    solid when its minimum-image distance to a centre is < radius. Returns solid[a,a,a]."""
    R = a * np.sqrt(2.0) / 4.0 if radius is None else float(radius)
    g = np.arange(a, dtype=np.float64)
    centres = np.array([[0.0, 0.0, 0.0], [a / 2, a / 2, 0.0], [a / 2, 0.0, a / 2], [0.0, a / 2, a / 2]])
    solid = np.zeros((a, a, a), dtype=bool)
    for cx, cy, cz in centres:
        dx = np.abs(g - cx)
        dx = np.minimum(dx, a - dx)
        dy = np.abs(g - cy)
        dy = np.minimum(dy, a - dy)
        dz = np.abs(g - cz)
        dz = np.minimum(dz, a - dz)
        solid |= (dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2) < R * R
    return solid.astype(np.uint8)


def random_spheres(shape, radius, porosity: float, seed: int, max_spheres: int = 10_000_000):
    """Overlapping solid spheres with seeded uniform centres, added one at a time until
    the fluid fraction is at or below `porosity`. `radius` is a number or a sequence of
    integer radii drawn uniformly per sphere. A node is solid when its periodic
    (minimum-image) squared distance to a centre is <= R^2. shape = (nz, ny, nx).
    Returns (solid uint8[nz,ny,nx], number of spheres)."""
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    solid = np.zeros(shape, dtype=np.uint8)
    total = nx * ny * nz
    n_solid = 0
    radii = np.atleast_1d(np.asarray(radius))
    target_solid = (1.0 - porosity) * total
    count = 0
    flat = solid.reshape(-1)
    while n_solid < target_solid and count < max_spheres:
        c = rng.uniform(0.0, 1.0, size=3) * np.array([nx, ny, nz], dtype=np.float64)
        R = float(radii[rng.integers(0, len(radii))]) if len(radii) > 1 else float(radii[0])
        r = int(np.ceil(R))
        xs = np.arange(int(np.floor(c[0])) - r, int(np.floor(c[0])) + r + 2)
        ys = np.arange(int(np.floor(c[1])) - r, int(np.floor(c[1])) + r + 2)
        zs = np.arange(int(np.floor(c[2])) - r, int(np.floor(c[2])) + r + 2)
        d2 = ((zs - c[2])[:, None, None] ** 2 + (ys - c[1])[None, :, None] ** 2
              + (xs - c[0])[None, None, :] ** 2)
        zz, yy, xx = np.broadcast_arrays(np.mod(zs, nz)[:, None, None],
                                         np.mod(ys, ny)[None, :, None],
                                         np.mod(xs, nx)[None, None, :])
        inside = d2 <= R * R
        lin = np.unique((zz[inside].astype(np.int64) * ny + yy[inside]) * nx + xx[inside])
        n_solid += int(np.count_nonzero(flat[lin] == 0))
        flat[lin] = 1
        count += 1
    return solid, count


def poiseuille_profile(H: int, u_max: float) -> np.ndarray:
    """Parabolic slit profile u_x(z) with the walls half way between the solid and the
    first fluid plane (z = 1/2 and z = H + 1/2), for z = 0..H+1 (zero on the solid planes)."""
    z = np.arange(H + 2, dtype=np.float64)
    u = 4.0 * u_max * (z - 0.5) * (H + 0.5 - z) / (H * H)
    u[0] = 0.0
    u[H + 1] = 0.0
    return u


def slit_flow(nx: int, ny: int, H: int, u_max: float) -> np.ndarray:
    """Velocity field u[3, H+2, ny, nx] of a parabolic slit flow along x."""
    u = np.zeros((3, H + 2, ny, nx))
    u[0] = poiseuille_profile(H, u_max)[:, None, None]
    return u


def random_flow(solid: np.ndarray, amplitude: float, seed: int) -> np.ndarray:
    """Seeded random velocity field u[3, ...], uniform in [-amplitude, amplitude] per
    component, zero on solid nodes (a test input, not a solution of any flow problem)."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(-amplitude, amplitude, size=(3,) + solid.shape)
    u[:, solid.astype(bool)] = 0.0
    return u


def drift_flow(solid: np.ndarray, mean: float, amplitude: float, seed: int) -> np.ndarray:
    """Seeded test flow u[3, ...]: random_flow(solid, amplitude, seed) plus a uniform drift
    `mean` along x on the fluid nodes (zero on solids), so that the mean fluid velocity is
    `mean` along x up to the sampling noise. A test input, not a solution of a flow problem."""
    u = random_flow(solid, amplitude, seed)
    u[0][solid == 0] += mean
    return u


def species(n: int, seed: int, D_b=(0.01, 0.1), k=(1e-4, 1e-1)):
    """n tracer species: D_b uniform in D_b, k_a and k_d log-uniform in k.
    Returns three float64 arrays (D_b, k_a, k_d)."""
    rng = np.random.default_rng(seed)
    Db = rng.uniform(D_b[0], D_b[1], size=n)
    lo, hi = np.log(k[0]), np.log(k[1])
    ka = np.exp(rng.uniform(lo, hi, size=n))
    kd = np.exp(rng.uniform(lo, hi, size=n))
    return Db, ka, kd
