"""Pins of the oracle's BGK lattice-Boltzmann solve (Eq. lb_evolution with a BGK collision,
the Guo body force and halfway bounce-back), against the mathematics of the scheme:
mass conservation, rest, and the exact discrete Stokes balance of a steady slit flow."""
import numpy as np

import oracle
from paper_1303_2470_gb300 import media


def test_mass_is_conserved_and_rest_stays_at_rest():
    rng = np.random.default_rng(1)
    solid = (rng.random((6, 5, 7)) < 0.25).astype(np.uint8)
    fluid = solid == 0
    f = oracle.lb_init(solid)
    m0 = f[:, fluid].sum()
    g = f.copy()
    for _ in range(30):
        g, u = oracle.lb_step(solid, g, (0.0, 0.0, 0.0), 1.0)
    assert np.max(np.abs(u)) < 1e-15
    assert np.allclose(g[:, fluid], f[:, fluid], rtol=0, atol=1e-16)
    # with a body force and a random start, mass is still conserved to rounding
    u0 = media.random_flow(solid, 0.02, seed=3)
    g = oracle.lb_init(solid, u0)
    m0 = g[:, fluid].sum()
    for _ in range(30):
        g, u = oracle.lb_step(solid, g, (1e-4, -2e-5, 3e-5), 0.9)
    assert abs(g[:, fluid].sum() - m0) < 1e-12 * m0


def test_slit_poiseuille_is_the_discrete_stokes_solution():
    """Steady unidirectional flow: every interior plane satisfies nu (u_{z+1} - 2 u_z +
    u_{z-1}) = -F with nu = (tau - 1/2)/3, so the profile is the parabola with walls half
    way plus a uniform slip; transverse components vanish."""
    H = 16
    for tau in (1.0, 0.8):
        nu = (tau - 0.5) / 3.0
        F = 8 * nu * 0.05 / H ** 2
        solid = media.slit(3, 3, H)
        u, steps, res, conv = oracle.lb_steady(solid, (F, 0, 0), tau, 1e-15, 60000, 200)
        ux = u[0, :, 1, 1]
        d2 = ux[3:H] - 2 * ux[2:H - 1] + ux[1:H - 2]
        assert np.max(np.abs(nu * d2 / (-F) - 1.0)) < 1e-9
        z = np.arange(H + 2)
        parab = F / (2 * nu) * (z - 0.5) * (H + 0.5 - z)
        slip = ux[1:H + 1] - parab[1:H + 1]
        assert np.ptp(slip) < 1e-9 * 0.05
        assert np.allclose(ux[1:H + 1], ux[H:0:-1], rtol=0, atol=1e-13)   # symmetric
        assert np.max(np.abs(u[1:])) < 1e-13
        assert np.allclose(u[:, 0], 0) and np.allclose(u[:, H + 1], 0)


def _duct(H):
    s = np.zeros((H + 2, H + 2, 3), np.uint8)   # square duct along x: walls at y, z = 0, H + 1
    s[0] = s[H + 1] = 1
    s[:, 0] = s[:, H + 1] = 1
    return s


def _duct_series(H, F, nu, terms=401):
    """Continuum Poiseuille flow in a square duct of side H with the walls half way between
    the solid and the first fluid nodes: nu lap u = -F, u = 0 on the walls, as the double
    sine series u = sum_{m,n odd} 16 F H^2 / (nu pi^4 m n (m^2 + n^2)) sin(m pi Y/H)
    sin(n pi Z/H) at the fluid nodes Y, Z = j - 1/2, j = 1..H. Returns u[Z, Y]."""
    Y = np.arange(1, H + 1) - 0.5
    m = np.arange(1, terms + 1, 2)
    sm = np.sin(np.outer(m, Y) * np.pi / H)
    A = 16 * F * H ** 2 / (nu * np.pi ** 4 * np.outer(m, m) * (m[:, None] ** 2 + m[None, :] ** 2))
    return np.einsum("mn,my,nz->zy", A, sm, sm)


def test_square_duct_converges_to_the_continuum_series():
    """Walls normal to y and z at once (the slit test only has z-walls): the steady flow
    keeps the duct's symmetries exactly and approaches the continuum series at second order
    in the resolution (halfway bounce-back), |error| / u_max below 0.6 / H^2."""
    nu, errs = 1.0 / 6.0, {}
    for H in (12, 24):
        F = 0.01 * nu / (0.0737 * H * H)             # u_max ~ 0.01 (square duct: 0.0737 F H^2 / nu)
        u, steps, res, conv = oracle.lb_steady(_duct(H), (F, 0, 0), 1.0, 1e-14, 400000, 100)
        assert conv
        ux = u[0, 1:H + 1, 1:H + 1, 1]
        scale = np.abs(ux).max()
        assert np.max(np.abs(ux - ux.T)) < 1e-12 * scale                   # y <-> z
        assert np.max(np.abs(ux - ux[::-1, :])) < 1e-12 * scale            # z -> H + 1 - z
        assert np.max(np.abs(ux - ux[:, ::-1])) < 1e-12 * scale            # y -> H + 1 - y
        assert np.max(np.abs(u[0] - u[0, :, :, :1])) < 1e-13               # invariant along x
        assert np.abs(u[1:]).max() < 1e-4 * scale
        ref = _duct_series(H, F, nu)
        errs[H] = np.max(np.abs(ux - ref)) / ref.max()
        assert errs[H] < 0.6 / H ** 2
    assert errs[12] / errs[24] > 3.0


def test_steady_criterion_and_step_budget():
    """lb_steady stops at the first checked step whose residual max|u(t) - u(t-1)| is
    below tol (a multiple of check_every), and reports non-convergence at max_steps."""
    H, nu = 32, 1.0 / 6.0
    F = 8 * nu * 0.05 / H ** 2          # u_max = 0.05 at tau = 1 (the slit flow config)
    solid = media.slit(2, 2, H)
    u, steps, res, conv = oracle.lb_steady(solid, (F, 0, 0), 1.0, 1e-7, 100000, 100)
    assert conv and res < 1e-7 and steps % 100 == 0
    assert abs(u[0].max() - 0.05) < 2e-3
    u2, steps2, res2, conv2 = oracle.lb_steady(solid, (F, 0, 0), 1.0, 1e-7, steps - 100, 100)
    assert not conv2 and steps2 == steps - 100 and res2 >= 1e-7


def _periodic_d3q19_components(solid):
    """Connected components of the fluid nodes under the 18 D3Q19 links (periodic), by
    scipy's graph routine: an implementation independent of the oracle's search."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    nz, ny, nx = solid.shape
    idx = np.arange(solid.size).reshape(solid.shape)
    fluid = solid == 0
    rows, cols = [], []
    for c in [(a, b, d) for a in (-1, 0, 1) for b in (-1, 0, 1) for d in (-1, 0, 1)
              if 1 <= abs(a) + abs(b) + abs(d) <= 2]:
        nb = np.roll(idx, shift=(-c[2], -c[1], -c[0]), axis=(0, 1, 2))
        ok = fluid & fluid.reshape(-1)[nb]
        rows.append(idx[ok])
        cols.append(nb[ok])
    r, c = np.concatenate(rows), np.concatenate(cols)
    g = coo_matrix((np.ones(r.size), (r, c)), shape=(solid.size, solid.size))
    _, lab = connected_components(g, directed=False)
    return lab.reshape(solid.shape)


def test_largest_cluster_matches_graph_components():
    for seed, (shape, R, phi) in enumerate([((12, 14, 10), 2, 0.45), ((20, 20, 20), 3, 0.35),
                                            ((9, 11, 13), 1.5, 0.5)]):
        solid, _ = media.random_spheres(shape, R, phi, seed=seed + 21)
        inc, size = oracle.largest_cluster(solid)
        lab = _periodic_d3q19_components(solid)
        fl = solid == 0
        sizes = np.bincount(lab[fl])
        assert size == sizes.max()
        best = [l for l in np.unique(lab[fl]) if sizes[l] == sizes.max()]
        # ties go to the cluster holding the smallest node index
        first = min(best, key=lambda l: np.flatnonzero((lab == l).reshape(-1) & fl.reshape(-1))[0])
        assert np.array_equal(inc.astype(bool), fl & (lab == first))


def test_sealed_pockets_stay_at_rest_and_the_flow_converges():
    """A channel plus a sealed single-node pocket and a sealed two-node pocket: the force acts
    on the channel only, the pockets keep u = 0 exactly, and the residual falls below tol
    (with the force on a one-node pocket its velocity would flip sign every step)."""
    solid = np.ones((9, 9, 12), dtype=np.uint8)
    solid[2:6, 2:6, :] = 0                 # channel along x, periodic
    solid[7, 7, 3] = 0                     # sealed single node
    solid[7, 1, 5:7] = 0                   # sealed pair along x
    inc, size = oracle.largest_cluster(solid)
    assert size == 16 * 12 and inc[7, 7, 3] == 0 and inc[7, 1, 5] == 0
    u, steps, res, conv = oracle.lb_steady(solid, (1e-5, 0, 0), tol=1e-12, max_steps=20000, check_every=50)
    assert conv and res < 1e-12
    assert np.all(u[:, 7, 7, 3] == 0.0) and np.all(u[:, 7, 1, 5:7] == 0.0)
    assert u[0, 4, 4, 0] > 0


def test_porous_medium_reaches_the_steady_criterion():
    """Random spheres (40^3, R = 6, porosity 0.40) at a force giving mean u ~ 0.01: with the
    two-iterate mean at failed checks the residual falls below 1e-7 (without it a period-2
    cycle at confined nodes keeps the residual near |F|), and the state it stops at is steady
    under the plain iteration: continuing plain BGK steps from the final populations (not a
    restart from an equilibrium), every node's one-step change max|u(t+1) - u(t)| stays
    below the tolerance at every one of 300 steps, and decays (no undamped oscillation is
    left: the largest change of the last 100 steps is below 0.6 of the first 100's)."""
    solid, _ = media.random_spheres((40, 40, 40), 6, 0.40, 3)
    F = (1.83e-3, 0.0, 0.0)
    tol = 1e-7
    u, steps, res, conv, f = oracle.lb_steady(solid, F, tol=tol, max_steps=20000, check_every=100, with_f=True)
    assert conv and res < tol and steps <= 5000
    fl = solid == 0
    assert 0.005 < u[0][fl].mean() < 0.02
    inc, _ = oracle.largest_cluster(solid)
    prev, change = u, []
    for _ in range(300):
        f, u2 = oracle.lb_step(solid, f, F, 1.0, forced=inc)
        change.append(np.abs(u2 - prev)[:, fl].max())
        prev = u2
    change = np.array(change)
    assert change.max() < tol
    assert change[-100:].max() < 0.6 * change[:100].max()


def test_density_start_and_output_conserve_each_regions_mass():
    """Eq. lb_evolution conserves the mass of every connected fluid region (streaming with
    bounce-back moves it, the collision and the Guo term keep it). From rest the final density
    of the forced channel sums to its node count and the sealed pockets keep density 1; a start
    f^eq(rho*, u*) from the converged state stays at that flow (and needs no more steps than
    from rest); a constant density offset in the start is the steady density's."""
    solid = np.ones((9, 9, 12), dtype=np.uint8)
    solid[2:6, 2:6, :] = 0
    solid[7, 7, 3] = 0
    solid[7, 1, 5:7] = 0
    inc, _ = oracle.largest_cluster(solid)
    ch = inc.astype(bool)
    pockets = (solid == 0) & ~ch
    F = (1e-5, 0.0, 0.0)
    u, steps, res, conv, rho = oracle.lb_steady(solid, F, tol=1e-12, max_steps=20000, check_every=50, with_rho=True)
    assert conv
    assert abs(rho[ch].sum() - ch.sum()) < 1e-10
    assert np.max(np.abs(rho[pockets] - 1.0)) < 1e-14
    assert np.all(rho[solid.astype(bool)] == 0.0)
    u2, s2, _, c2, rho2 = oracle.lb_steady(solid, F, tol=1e-12, max_steps=20000, check_every=50, u_init=u,
                                            rho_init=rho, with_rho=True)
    assert c2 and s2 <= steps
    assert np.max(np.abs(u2 - u)) < 1e-9 * np.abs(u).max()
    r0 = np.where(ch, 1.01, 1.0)
    _, _, _, c3, rho3 = oracle.lb_steady(solid, F, tol=1e-12, max_steps=20000, check_every=50, rho_init=r0,
                                         with_rho=True)
    assert c3 and abs(rho3[ch].mean() - 1.01) < 1e-12
