"""The seeded input generators (paper_1303_2470_gb300/media.py) against brute-force
restatements of their definitions and the geometry they claim (CPU).

These generators feed both the GPU library and the oracle, so a mistake here would pass
every parity test unnoticed: each recipe is checked on its own.
"""
import itertools

import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

from paper_1303_2470_gb300 import media

# the 18 moving D3Q19 links (faces and edges of the unit cube)
LINKS = [c for c in itertools.product((-1, 0, 1), repeat=3) if 1 <= sum(map(abs, c)) <= 2]


def _fluid_clusters(solid):
    """Connected components of the fluid nodes under periodic D3Q19 links."""
    nz, ny, nx = solid.shape
    idx = np.arange(solid.size).reshape(solid.shape)
    fluid = solid == 0
    rows, cols = [], []
    for cx, cy, cz in LINKS:
        nb = np.roll(idx, shift=(-cz, -cy, -cx), axis=(0, 1, 2))
        both = fluid & np.roll(fluid, shift=(-cz, -cy, -cx), axis=(0, 1, 2))
        rows.append(idx[both])
        cols.append(nb[both])
    r, c = np.concatenate(rows), np.concatenate(cols)
    g = coo_matrix((np.ones(r.size, dtype=np.int8), (r, c)), shape=(solid.size, solid.size))
    _, labels = connected_components(g, directed=False)
    return np.unique(labels[fluid.reshape(-1)]).size


def _min_image_mask(shape, centres, radii, strict):
    """Solid mask by brute force: node (x, y, z) is solid when, for some centre, the
    smallest distance over all periodic images is below R (strict) or at most R."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    solid = np.zeros(shape, dtype=bool)
    for (cx, cy, cz), R in zip(centres, radii):
        best = np.full(shape, np.inf)
        for ix, iy, iz in itertools.product((-1, 0, 1), repeat=3):
            d2 = (x - cx - ix * nx) ** 2 + (y - cy - iy * ny) ** 2 + (z - cz - iz * nz) ** 2
            best = np.minimum(best, d2)
        solid |= (best < R * R) if strict else (best <= R * R)
    return solid.astype(np.uint8)


def test_slit_and_bulk():
    s = media.slit(5, 4, 7)
    assert s.shape == (9, 4, 5) and s.dtype == np.uint8
    assert s[0].all() and s[8].all() and not s[1:8].any()
    b = media.bulk(3, 4, 5)
    assert b.shape == (5, 4, 3) and not b.any()


@pytest.mark.parametrize("a", [12, 16, 20])
def test_fcc_cell_is_the_minimum_image_rule_at_the_corner_and_face_centres(a):
    R = a * np.sqrt(2.0) / 4.0
    centres = [(0, 0, 0), (a / 2, a / 2, 0), (a / 2, 0, a / 2), (0, a / 2, a / 2)]
    ref = _min_image_mask((a, a, a), centres, [R] * 4, strict=True)
    assert np.array_equal(media.fcc(a), ref)
    # a smaller radius as well
    ref = _min_image_mask((a, a, a), centres, [0.3 * a] * 4, strict=True)
    assert np.array_equal(media.fcc(a, radius=0.3 * a), ref)


def test_fcc_cell_symmetry_contact_points_and_connected_pore_space():
    a = 100
    s = media.fcc(a)
    # cubic symmetry: every permutation of the axes and every mirror maps the cell to itself
    for perm in itertools.permutations(range(3)):
        assert np.array_equal(s, s.transpose(perm))
    for ax in range(3):
        assert np.array_equal(s, np.roll(np.flip(s, axis=ax), 1, axis=ax))
    # touching spheres meet at the midpoint between a corner and a face centre, at distance
    # exactly R from both: fluid under the strict rule
    assert s[0, a // 4, a // 4] == 0 and s[a // 4, 0, a // 4] == 0
    # porosity tends to the continuum value 1 - pi / (3 sqrt 2) of the compact packing
    phi = 1.0 - s.mean()
    assert abs(phi - (1.0 - np.pi / (3.0 * np.sqrt(2.0)))) < 5e-3
    # the pore space is one D3Q19-connected cluster (the body force and tracers reach it all)
    assert _fluid_clusters(s) == 1


def test_fcc_porosity_converges_with_resolution():
    exact = 1.0 - np.pi / (3.0 * np.sqrt(2.0))
    gaps = [abs(1.0 - media.fcc(a).mean() - exact) for a in (24, 48, 96)]
    assert gaps[2] < gaps[0] and gaps[2] < 5e-3


@pytest.mark.parametrize("shape,radius,phi,seed", [((16, 20, 24), 3, 0.6, 4), ((18, 18, 18), [2, 3, 4], 0.45, 9),
                                                   ((10, 12, 14), 2.5, 0.7, 1)])
def test_random_spheres_is_the_union_of_its_seeded_spheres(shape, radius, phi, seed):
    solid, count = media.random_spheres(shape, radius, phi, seed)
    # replay the generator's draws: per sphere three uniform centre coordinates (x, y, z),
    # then a radius index when several radii are given
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    radii = np.atleast_1d(np.asarray(radius, dtype=np.float64))
    centres, rs = [], []
    for _ in range(count):
        c = rng.uniform(0.0, 1.0, size=3) * np.array([nx, ny, nz], dtype=np.float64)
        R = float(radii[rng.integers(0, len(radii))]) if len(radii) > 1 else float(radii[0])
        centres.append(tuple(c))
        rs.append(R)
    assert np.array_equal(solid, _min_image_mask(shape, centres, rs, strict=False))
    # it stops at the first sphere that brings the fluid fraction to the target or below
    fluid = 1.0 - solid.mean()
    assert fluid <= phi
    without_last = _min_image_mask(shape, centres[:-1], rs[:-1], strict=False)
    assert 1.0 - without_last.mean() > phi


def test_random_spheres_is_seeded():
    a, n1 = media.random_spheres((20, 20, 20), 3, 0.5, seed=3)
    b, n2 = media.random_spheres((20, 20, 20), 3, 0.5, seed=3)
    c, _ = media.random_spheres((20, 20, 20), 3, 0.5, seed=4)
    assert n1 == n2 and np.array_equal(a, b) and not np.array_equal(a, c)


def test_poiseuille_profile_and_slit_flow():
    for H in (5, 8, 33):
        u = media.poiseuille_profile(H, 0.05)
        assert u.shape == (H + 2,) and u[0] == 0.0 and u[H + 1] == 0.0
        assert np.allclose(u, u[::-1], rtol=0, atol=1e-15)           # symmetric about the mid-plane
        z = np.arange(1, H + 1, dtype=np.float64)
        # the parabola vanishing half-way between the solid and the first fluid plane
        assert np.allclose(u[1:H + 1], 0.05 * 4 * (z - 0.5) * (H + 0.5 - z) / H ** 2, rtol=1e-14, atol=0)
        assert (u[1:H + 1] > 0).all() and u.max() <= 0.05 * (1 + 1e-12)
    u = media.poiseuille_profile(7, 0.03)
    assert u[4] == pytest.approx(0.03, rel=1e-14)                    # odd H: the mid-plane is a node
    f = media.slit_flow(4, 3, 7, 0.03)
    assert f.shape == (3, 9, 3, 4)
    assert np.array_equal(f[0], np.broadcast_to(u[:, None, None], (9, 3, 4))) and not f[1:].any()


def test_random_flow_and_species():
    solid, _ = media.random_spheres((12, 12, 12), 2, 0.6, seed=2)
    u = media.random_flow(solid, 0.02, seed=7)
    assert u.shape == (3, 12, 12, 12)
    assert not u[:, solid.astype(bool)].any() and np.abs(u).max() <= 0.02
    assert np.array_equal(u, media.random_flow(solid, 0.02, seed=7))
    Db, ka, kd = media.species(20000, seed=5)
    assert Db.min() >= 0.01 and Db.max() <= 0.1
    for k in (ka, kd):
        assert k.min() >= 1e-4 and k.max() <= 1e-1
        # log-uniform: the mean of log k is the midpoint (5 standard errors)
        lo, hi = np.log(1e-4), np.log(1e-1)
        assert abs(np.log(k).mean() - 0.5 * (lo + hi)) < 5 * (hi - lo) / np.sqrt(12 * k.size)
    assert abs(Db.mean() - 0.055) < 5 * 0.09 / np.sqrt(12 * Db.size)
    Db2, ka2, kd2 = media.species(20000, seed=5)
    assert np.array_equal(Db, Db2) and np.array_equal(ka, ka2) and np.array_equal(kd, kd2)
