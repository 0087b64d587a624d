"""An independent derivation of the slit's wall-normal D(t), used only to pin the oracle's
continuum module (oracle/continuum.py), which follows the paper's printed Eq. exact_D.

Derived here from the model itself (advection-diffusion without flow and the surface
exchange of Sec. Model): a tracer diffuses with D_b in x in [-L/2, L/2]; at a wall it
adsorbs at rate k_a (length/time) per unit density and desorbs at rate k_d. With the
equilibrium start (free density 1/(L + 2K) on the fluid, K = k_a/k_d adsorbed at each wall)
the position autocorrelation is C(t) = <x(0) x(t)> and D(t) = -dC/dt. The conditional mean
u(x,t) = E[x(t) | x(0) = x] solves du/dt = D_b u'' with D_b du/dn = k_a (v - u) at a wall,
where the adsorbed mean obeys dv/dt = k_d (u - v), u(x,0) = x, v(0) = +-L/2. In Laplace space
(chi = sqrt(s/D_b), kappa = chi L/2):
    u(x) = x/s + A sinh(chi x),
    A = -(D_b/s)(s + k_d) / [D_b chi (s + k_d) cosh kappa + k_a s sinh kappa],
    C(s) = [L^3/(12 s) + 2A ((L/2) cosh kappa / chi - sinh kappa / chi^2) + K L v(s)] / (L + 2K),
    v(s) = (L/2 + k_d u(L/2)) / (s + k_d),     D(s) = C(0) - s C(s),
    C(0) = [L^3/12 + K L^2/2] / (L + 2K).
It is evaluated with mpmath (arbitrary precision, its own Talbot inversion), so neither the
algebra nor the inversion is shared with the oracle.
"""
from __future__ import annotations

import numpy as np


def slit_D_laplace(s, L, D_b, k_a, k_d):
    """D-hat(s) of the wall-normal D(t) (mpmath arithmetic)."""
    import mpmath as mm
    K = mm.mpf(0) if k_a == 0 else mm.mpf(k_a) / mm.mpf(k_d)
    chi = mm.sqrt(s / D_b)
    kap = chi * L / 2
    ch, sh = mm.cosh(kap), mm.sinh(kap)
    A = -(D_b / s) * (s + k_d) / (D_b * chi * (s + k_d) * ch + k_a * s * sh)
    u_wall = L / (2 * s) + A * sh
    v = (L / 2 + k_d * u_wall) / (s + k_d)
    C = (L ** 3 / (12 * s) + 2 * A * ((L / 2) * ch / chi - sh / chi ** 2) + K * L * v) / (L + 2 * K)
    C0 = (mm.mpf(L) ** 3 / 12 + K * mm.mpf(L) ** 2 / 2) / (L + 2 * K)
    return C0 - s * C


def slit_D(ts, L, D_b, k_a, k_d, dps=30):
    """D(t) at the times ts > 0 by mpmath's Talbot inversion of slit_D_laplace."""
    import mpmath as mm
    mm.mp.dps = dps
    f = lambda s: slit_D_laplace(s, mm.mpf(L), mm.mpf(D_b), mm.mpf(k_a), mm.mpf(k_d))  # noqa: E731
    return np.array([float(mm.invertlaplace(f, float(t), method="talbot")) for t in ts])


def slit_D_no_sorption(ts, L, D_b, nterms=2000):
    """Pure diffusion between reflecting walls: D(t) = sum over odd n of
    8 D_b/(n pi)^2 exp(-D_b (n pi/L)^2 t) (the textbook eigenfunction series of the
    position autocorrelation)."""
    n = np.arange(1, 2 * nterms, 2)[:, None]
    return (8 * D_b / (n * np.pi) ** 2 * np.exp(-D_b * (n * np.pi / L) ** 2 * np.asarray(ts)[None, :])).sum(0)


def slowest_rate(L, D_b, k_a, k_d):
    """Decay rate sigma_1 = D_b beta_1^2 of the slowest odd (wall-normal) mode: the smallest
    root beta in (0, pi/L) of (k_d - D_b beta^2) cos(beta L/2) - k_a beta sin(beta L/2) = 0,
    the zero of the transform's denominator at s = -D_b beta^2."""
    from scipy.optimize import brentq
    f = lambda b: (k_d - D_b * b * b) * np.cos(b * L / 2) - k_a * b * np.sin(b * L / 2)  # noqa: E731
    b = brentq(f, 1e-12, np.pi / L, xtol=1e-300, rtol=1e-15, maxiter=500)
    return D_b * b * b
