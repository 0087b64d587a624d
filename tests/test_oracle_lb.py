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
