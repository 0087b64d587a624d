"""Continuum exact solutions the paper validates its lattice method against (Sec. Validation).

Test infrastructure, like the rest of oracle/: only the tests, the smoke check and the
benchmark's CPU legs may import it. Plain numpy, FP64.

  * slit_D_hat / slit_D  -- Eq. exact_D: wall-normal D(t) of tracers between two sorbing
    walls a distance L apart, as a Laplace transform and its numerical inverse;
  * adsorbed_fraction    -- Eq. fa;
  * taylor_aris_K        -- Eq. exact_K: Taylor-Aris dispersion along a Poiseuille flow;
  * log_fit              -- the slope and origin of the linear fit of log10 D(t) the paper
    uses to quantify its errors (Fig. 2).

Readings of the printed equations:
  * Eq. exact_D prints D(t)/D_b on its left side, but the right side already carries the
    dimensions of a diffusion coefficient (the bracket is [length^3/time] in the Laplace
    domain, divided by 2k_a + k_d L [length/time]); at t = 0+ it gives (1 - f_a) D_b, the
    mobile fraction times D_b, only when read as D(t). It is read as D(t) here. Pinned in
    the tests against a transform derived independently from the model's diffusion and
    sorption equations, the pure-diffusion eigenfunction series, the mobile-fraction start
    and the decay rate of the slowest wall-normal mode.
  * Eq. exact_K prints a leading 1; at Pe = 0 the formula must reduce to the plateau
    1/(1 + 2y) of a sorbing slit, so the leading term is read as 1/(1 + 2y) (the printed form
    is available as leading="printed").
"""
from __future__ import annotations

import numpy as np


def _tanh(kappa):
    """tanh of complex arguments with Re >= 0, without overflow for large |kappa|."""
    e = np.exp(-2.0 * kappa)
    return (1.0 - e) / (1.0 + e)


def slit_D_hat(s, L, D_b, k_a, k_d):
    """Laplace transform of D(t) (Eq. exact_D, read as D(t)), chi = sqrt(s/D_b),
    kappa = chi L/2, written with tanh(kappa) (numerator and denominator of the second
    term divided by cosh kappa). With k_a = 0 the k_d factors cancel and the limit
    D_b/s - 2 tanh(kappa)/(L chi^3) (pure diffusion between reflecting walls) is used."""
    s = np.asarray(s, dtype=np.complex128)
    chi = np.sqrt(s / D_b)
    th = _tanh(chi * L / 2.0)
    if k_a == 0.0:
        return D_b / s - 2.0 * th / (L * chi ** 3)
    second = 2.0 * k_d * (k_d + s) * th / (chi ** 3 * ((k_d + s) + k_a * chi * th))
    return (k_d * L * D_b / s - second) / (2.0 * k_a + k_d * L)


def invert_laplace(F, t, M=20):
    """f(t) from its transform F by the fixed-Talbot contour of Abate and Valko (2004):
    r = 2M/(5t), theta_k = k pi/M, s_k = r theta_k (cot theta_k + i),
    sigma_k = theta_k + (theta_k cot theta_k - 1) cot theta_k,
    f(t) ~ (r/M) [F(r) e^(rt)/2 + sum_{k=1}^{M-1} Re(e^(t s_k) F(s_k) (1 + i sigma_k))].
    In double precision M = 20 gives about 7 significant digits on these transforms."""
    k = np.arange(1, M)
    th = k * np.pi / M
    cot = 1.0 / np.tan(th)
    r = 2.0 * M / (5.0 * t)
    s = r * th * (cot + 1j)
    sig = th + (th * cot - 1.0) * cot
    head = 0.5 * np.exp(r * t) * F(np.complex128(r)).real
    return r / M * (head + np.sum((np.exp(t * s) * F(s) * (1.0 + 1j * sig)).real))


def slit_D(ts, L, D_b, k_a, k_d, M=20):
    """Continuum wall-normal D(t) of Eq. exact_D at the times ts > 0."""
    F = lambda s: slit_D_hat(s, L, D_b, k_a, k_d)  # noqa: E731
    return np.array([invert_laplace(F, float(t), M) for t in np.atleast_1d(ts)])


def adsorbed_fraction(L, k_a, k_d):
    """Eq. fa: fraction of tracers adsorbed at equilibrium in a slit of width L."""
    if k_a == 0.0:
        return 0.0
    return 1.0 / (1.0 + k_d * L / (2.0 * k_a))


def taylor_aris_K(Pe, y, D_b, L, k_d, leading="read"):
    """Eq. exact_K: K for Poiseuille flow in a sorbing slit, Pe = L vbar/D_b, y = k_a/(k_d L).
    leading="read" uses 1/(1+2y) as the leading term, "printed" the printed 1."""
    lead = 1.0 if leading == "printed" else 1.0 / (1.0 + 2.0 * y)
    extra = 0.0 if y == 0.0 else (D_b / (L * L * k_d)) * 2.0 * y / (1.0 + 2.0 * y) ** 3
    return D_b * (lead + Pe ** 2 * ((102.0 * y * y + 18.0 * y + 1.0) / (210.0 * (1.0 + 2.0 * y) ** 3) + extra))


def log_fit(ts, D):
    """Least-squares line through log10 D(t) against t: (slope, origin)."""
    slope, origin = np.polyfit(np.asarray(ts, dtype=np.float64), np.log10(np.asarray(D, dtype=np.float64)), 1)
    return float(slope), float(origin)
