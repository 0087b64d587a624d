"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every expected value comes from a closed
form derived from the paper's equations, from a number printed in the paper
(tests/golden/paper_printed.json), from an independent Markov-chain restatement of the
method (tests/_chains.py: dense chain, exact z-chain of a slit, random walkers), or from a
lattice identity. A dropped term, a wrong sign or index, or a transposed operand in the
oracle fails at least one of these.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import continuum as oc
import _chains as chains
from paper_1303_2470_gb300 import media

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table_identities(c, w):
    c = np.asarray(c, dtype=np.float64)
    assert np.isclose(w.sum(), 1.0, atol=1e-15)
    assert np.allclose((w[:, None] * c).sum(0), 0.0, atol=1e-15)
    second = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(second, np.eye(3) / 3.0, atol=1e-15)          # c_s^2 = 1/3
    fourth = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.allclose(fourth, iso, atol=1e-15)


def test_d3q19_tables():
    c, w, opp = oracle.d3q19()
    _table_identities(c, w)
    assert np.all(c[opp] == -c)
    assert len({tuple(v) for v in c}) == 19
    # the chain restatement's table (moving links only, plus the rest weight 1/3)
    cc = np.vstack([[0, 0, 0], chains.C18])
    ww = np.concatenate([[1.0 / 3.0], chains.W18])
    _table_identities(cc, ww)


def test_bulk_box_diffuses_at_D_b():
    """No solid, fluid at rest: an unbiased random walk, D(t) = D_b for every t
    (D_b = lambda c_s^2 / 4 of Sec. Algorithm, so lambda = 12 D_b)."""
    for D_b in (0.01, 0.05, 1.0 / 12.0):
        p = oracle.Problem(media.bulk(5, 4, 6), None, D_b, 0.0, 0.0)
        r = oracle.run(p, g=0, nsteps=20)
        assert np.allclose(r.D, D_b, rtol=0, atol=1e-15)
        assert np.allclose(r.Z[1:], 0.0, atol=1e-17)


def test_uniform_flow_gives_K_equal_D_b():
    """Uniform flow in a periodic box: steps are iid with mean u, so Z(t>=1) = u_g^2,
    Z(0) = lambda/6 + u_g^2 and K = (Z0 - Zinf)/2 + sum (Z_m - Zinf) = D_b."""
    D_b = 0.05
    U = np.array([0.03, -0.02, 0.01])
    solid = media.bulk(4, 5, 3)
    u = np.broadcast_to(U[:, None, None, None], (3,) + solid.shape).copy()
    p = oracle.Problem(solid, u, D_b, 0.0, 0.0)
    for g in range(3):
        r = oracle.run(p, g=g, nsteps=10)
        assert np.isclose(r.Z[0], 2 * D_b + U[g] ** 2, rtol=0, atol=1e-15)
        assert np.allclose(r.Z[1:], U[g] ** 2, rtol=0, atol=1e-15)
        K = (r.Z[0] - U[g] ** 2) / 2 + np.sum(r.Z[1:] - U[g] ** 2)
        assert np.isclose(K, D_b, rtol=0, atol=1e-15)


@pytest.mark.slow
def test_slit_pure_diffusion_config():
    """8x8 periodic slit, H = 16 fluid planes, u = 0, D_b = 0.05, k_a = k_d = 0.01,
    density uniform over the fluid, 1e4 steps (the paper's pure-diffusion slit test).
      * total mass sum(P) + sum(Gamma) conserved to 1e-12 (reading R1 makes it exact);
      * Gamma/rho -> K = k_a/(k_d dx) at interfacial nodes (Sec. Algorithm weights);
      * final per-node density H/(H+2K) of the initial one;
      * lateral D_x(t) = D_b (H - 1/3)/(H + 2K) at every t (lattice closed form: with
        u = 0, Z_x(t>=1) = 0 by x-symmetry, and the wall planes lose the two blocked
        edge links of lateral variance, 1/6 of it)."""
    H, K, D_b = 16, 1.0, 0.05
    p = oracle.Problem(media.slit(8, 8, H), None, D_b, 0.01, 0.01)
    r = oracle.run(p, g=0, nsteps=10_000, init="uniform")
    total = r.mass_free + r.mass_ads
    assert np.max(np.abs(total - 1.0)) < 1e-12
    n_iface = 2 * 8 * 8
    gamma_over_rho = (r.mass_ads[-1] / n_iface) / (r.iface_free[-1] / n_iface)
    assert abs(gamma_over_rho - K) < 1e-10
    assert abs(r.mass_free[-1] - H / (H + 2 * K)) < 1e-10
    D_lattice = D_b * (H - 1.0 / 3.0) / (H + 2 * K)
    assert np.max(np.abs(r.D - D_lattice)) < 1e-12
    assert abs(D_lattice - 0.0435185185185185) < 1e-15


def test_slit_wall_normal_start_and_confinement():
    """Wall-normal D_z(0) = D_b (H - 1)/(H + 2K): the wall planes lose half of their
    normal variance (the five links into the wall). Under full confinement D_z(t) -> 0
    (Sec. Validation, slit discussion)."""
    H, D_b, ka, kd = 8, 0.05, 0.02, 0.01
    K = ka / kd
    p = oracle.Problem(media.slit(4, 4, H), None, D_b, ka, kd)
    r = oracle.run(p, g=2, nsteps=4000)
    assert abs(r.D[0] - D_b * (H - 1.0) / (H + 2 * K)) < 1e-15
    assert abs(r.D[-1]) < 1e-5 * r.D[0]
    late = r.D[2000:]
    assert np.all(np.diff(late) < 0) and np.all(late > 0)


def test_lateral_plateau_approaches_continuum_as_1_over_3H():
    """Lattice D_x = D_b (H-1/3)/(H+2K) vs the continuum D_b/(1+2K/H): the relative gap is
    -1/(3H) exactly, so it vanishes as the slit widens."""
    D_b, ka, kd = 0.05, 0.01, 0.01
    K = ka / kd
    for H in (16, 32, 64, 100):
        p = oracle.Problem(media.slit(3, 3, H), None, D_b, ka, kd)
        r = oracle.run(p, g=0, nsteps=0)
        cont = D_b / (1.0 + 2 * K / H)
        assert abs(r.D[0] / cont - 1.0 - (-1.0 / (3 * H))) < 1e-13


def test_paper_printed_adsorbed_fractions():
    """The paper prints f_a of about 16 %, 66 %, 95 % for L = 100, k_a = 0.1 and
    k_d = 1e-2, 1e-3, 1e-4 (Eq. fa). The oracle's Boltzmann weights on a slit with
    H = L fluid planes give the adsorbed share exactly (1 + k_d L/(2 k_a))^-1."""
    g = json.load(open(os.path.join(GOLDEN, "paper_printed.json")))["slit_adsorbed_fraction"]
    L, ka = g["L"], g["k_a"]
    for kd, printed in zip(g["k_d"], g["f_a_percent"]):
        p = oracle.Problem(media.slit(3, 3, L), None, g["D_b"], ka, kd)
        pi, pa = oracle.equilibrium(p)
        fa = pa.sum() / (pi.sum() + pa.sum())
        assert abs(fa - 1.0 / (1.0 + kd * L / (2 * ka))) < 1e-13
        assert round(100 * fa) == printed or abs(100 * fa - printed) < 1.0


def test_initial_D_is_mobile_fraction_times_D_b():
    """Sec. Validation: D(t=0) is the mobile fraction times D_b. On the lattice the wall
    planes lose 1/6 of their lateral variance, so D_x(0)/((1-f_a) D_b) = 1 - 1/(3H)."""
    g = json.load(open(os.path.join(GOLDEN, "paper_printed.json")))["slit_adsorbed_fraction"]
    L, ka = g["L"], g["k_a"]
    for kd in g["k_d"]:
        p = oracle.Problem(media.slit(3, 3, L), None, g["D_b"], ka, kd)
        r = oracle.run(p, g=0, nsteps=0)
        fa = 1.0 / (1.0 + kd * L / (2 * ka))
        assert abs(r.D[0] / ((1 - fa) * g["D_b"]) - (1 - 1.0 / (3 * L))) < 1e-13


@pytest.mark.parametrize("ka,kd", [(0.0, 0.0), (1e-3, 1e-2), (1e-2, 1e-3), (0.05, 0.02)])
def test_oracle_matches_exact_slit_chain(ka, kd):
    """Poiseuille slit with sorption: the 3D oracle's Z_g(t) equals that of the exact
    H+2-state reduction of the same chain, for g = x (flow) and z (wall-normal)."""
    H, D_b, umax = 10, 0.02, 0.05
    solid = media.slit(4, 3, H)
    u = media.slit_flow(4, 3, H, umax)
    p = oracle.Problem(solid, u, D_b, ka, kd)
    ch, pi0 = chains.z_chain(H, media.poiseuille_profile(H, umax), D_b, ka, kd)
    T = 300
    for g in (0, 2):
        r = oracle.run(p, g=g, nsteps=T - 1)
        Zc = chains.zchain_vacf(ch, pi0, g, T)
        assert np.max(np.abs(r.Z - Zc)) < 1e-14 * max(1.0, abs(Zc[0])) * 10


def test_oracle_matches_dense_chain_on_random_medium():
    """Random solid, random flow and sorption on a 6x5x7 lattice: Z_g(t) of the oracle equals
    the dense Markov chain's for all three directions, and the oracle's density and
    velocity-moment fields (free and adsorbed) equal the chain's state vectors."""
    rng = np.random.default_rng(7)
    solid = (rng.random((7, 5, 6)) < 0.2).astype(np.uint8)
    u = media.random_flow(solid, 0.03, seed=11)
    D_b, ka, kd = 0.04, 0.03, 0.02
    p = oracle.Problem(solid, u, D_b, ka, kd)
    ch, free, ads, pi0 = chains.dense_chain(solid, u, D_b, ka, kd)
    T = 40
    for g in range(3):
        r = oracle.run(p, g=g, nsteps=T - 1)
        Zc = ch.vacf(pi0, g, T)
        assert np.max(np.abs(r.Z - Zc)) < 1e-14
        # velocity moment field at t = T: pi0 V T^(T-1)
        w = pi0 @ (ch.T * ch.inc[g])
        for _ in range(T - 1):
            w = w @ ch.T
        fl = free >= 0
        assert np.allclose(r.Pg.reshape(-1)[fl], w[free[fl]], rtol=0, atol=1e-15)
        ia = ads >= 0
        assert np.allclose(r.Pga.reshape(-1)[ia], w[ads[ia]], rtol=0, atol=1e-15)
    # density field started at equilibrium and advanced T steps: pi0 T^T
    r = oracle.run(p, g=0, nsteps=T - 1, init="equilibrium")
    v = pi0.copy()
    for _ in range(T):
        v = v @ ch.T
    fl = free >= 0
    assert np.allclose(r.P.reshape(-1)[fl], v[free[fl]], rtol=0, atol=1e-15)
    ia = ads >= 0
    assert np.allclose(r.Pa.reshape(-1)[ia], v[ads[ia]], rtol=0, atol=1e-15)


@pytest.mark.slow
def test_random_walkers_reproduce_vacf():
    """Seeded random walkers on an 8^3 medium with flow and sorption (the Brownian picture
    the paper names as the alternative to MP): the sample <v_g(0) v_g(t)> agrees with the
    oracle's Z_g(t) within 4 standard errors, and the sample MSD increments give D(t) =
    [MSD(t+1) - MSD(t)]/2 (reading R5 of the time indexing)."""
    rng = np.random.default_rng(3)
    solid = (rng.random((8, 8, 8)) < 0.15).astype(np.uint8)
    u = media.random_flow(solid, 0.02, seed=5)
    D_b, ka, kd = 0.05, 0.05, 0.1
    p = oracle.Problem(solid, u, D_b, ka, kd)
    ch, free, ads, pi0 = chains.dense_chain(solid, u, D_b, ka, kd)
    T = 12
    steps = chains.walkers(ch, pi0, 1_000_000, T, seed=2024)
    for g in range(3):
        r = oracle.run(p, g=g, nsteps=T - 1)
        v0 = steps[0, g].astype(np.float64)
        for t in range(T + 1):
            prod = v0 * steps[t, g]
            se = prod.std() / np.sqrt(prod.size)
            assert abs(prod.mean() - r.Z[t]) < 4 * se + 1e-12


def test_stationary_slit_walkers_give_D_of_t():
    """Slit with Poiseuille flow (Boltzmann weights are stationary): the walkers' MSD
    increments equal 2 D(t) of the oracle within 4 standard errors."""
    H, D_b, ka, kd = 6, 0.05, 0.05, 0.1
    ch, pi0 = chains.z_chain(H, media.poiseuille_profile(H, 0.03), D_b, ka, kd)
    p = oracle.Problem(media.slit(4, 4, H), media.slit_flow(4, 4, H, 0.03), D_b, ka, kd)
    T = 10
    r = oracle.run(p, g=0, nsteps=T - 1)
    steps = chains.walkers(ch, pi0, 1_000_000, T, seed=99)[:, 0].astype(np.float64)
    vbar = float(pi0 @ ch.Vg[0].sum(1))
    dev = steps - vbar
    disp = np.cumsum(dev, axis=0)
    for t in range(T):
        # [MSD(t+1)-MSD(t)]/2 of the drift-free displacement = D(t) - t vbar^2 - vbar^2/2
        a = disp[t + 1] ** 2 - disp[t] ** 2
        est = a.mean() / 2.0
        se = a.std() / np.sqrt(a.size) / 2.0
        target = r.D[t + 1] - (t + 1) * vbar ** 2 - vbar ** 2 / 2.0
        assert abs(est - target) < 4 * se


@pytest.mark.parametrize("ka,kd", [(0.0, 0.0), (1e-3, 1e-2), (1e-2, 1e-3)])
def test_taylor_aris_dispersion_of_the_lattice_chain(ka, kd):
    """Eq. exact_K for Poiseuille flow in a slit, H = 32, D_b = 0.02, u_max = 0.05: the
    lattice K (exact, from the slit chain) agrees with the continuum formula within a few
    percent, and tends to it when the slit is refined at fixed Pe and y (the 1/(1+2y)
    leading term, reading R8). The 3D oracle's K after T steps equals the chain's."""
    D_b = 0.02
    errs = []
    for H in (32, 64):
        umax = 0.05 * 32 / H                      # keep Pe = L vbar / D_b fixed
        kd_H = kd * (32 / H) ** 2                 # keep y and the D_b/(L^2 k_d) term fixed
        ka_H = ka * (32 / H)
        ch, pi0 = chains.z_chain(H, media.poiseuille_profile(H, umax), D_b, ka_H, kd_H)
        K, _ = chains.zchain_K(ch, pi0, 0)
        y = 0.0 if ka == 0 else ka_H / (kd_H * H)
        vfluid = media.poiseuille_profile(H, umax)[1:H + 1].mean()   # mean flow velocity
        Pe = H * vfluid / D_b
        exact = oc.taylor_aris_K(Pe, y, D_b, H, kd_H if kd_H > 0 else 1.0, "read")
        errs.append(abs(K / exact - 1.0))
    assert errs[0] < 0.05
    assert errs[1] < errs[0]
    # 3D oracle vs chain on the H = 32 slit over a short window
    ch, pi0 = chains.z_chain(32, media.poiseuille_profile(32, 0.05), D_b, ka, kd)
    p = oracle.Problem(media.slit(3, 3, 32), media.slit_flow(3, 3, 32, 0.05), D_b, ka, kd)
    r = oracle.run(p, g=0, nsteps=199)
    assert np.max(np.abs(r.Z - chains.zchain_vacf(ch, pi0, 0, 200))) < 1e-14


def test_taylor_aris_refinement_selects_the_leading_term_reading():
    """Eq. exact_K prints a leading '1'; at Pe = 0 the formula must reduce to the lateral
    plateau 1/(1+2y) of a sorbing slit, so the leading term is read as 1/(1+2y) (R8).
    Refining the slit at fixed Pe and y, the lattice K's gap to the continuum (which falls
    like 1/H) extrapolates to zero under that reading and not under the printed one."""
    D_b, ka, kd = 0.02, 1e-2, 1e-3
    gaps = {"read": [], "printed": []}
    for H in (64, 128):
        umax, kd_H, ka_H = 0.05 * 32 / H, kd * (32 / H) ** 2, ka * (32 / H)
        ch, pi0 = chains.z_chain(H, media.poiseuille_profile(H, umax), D_b, ka_H, kd_H)
        K, _ = chains.zchain_K(ch, pi0, 0)
        y = ka_H / (kd_H * H)
        Pe = H * media.poiseuille_profile(H, umax)[1:H + 1].mean() / D_b
        for lead in gaps:
            gaps[lead].append(K / oc.taylor_aris_K(Pe, y, D_b, H, kd_H, lead) - 1.0)
    extrap = {lead: 2 * g[1] - g[0] for lead, g in gaps.items()}
    assert abs(extrap["read"]) < 1e-3
    assert abs(extrap["printed"]) > 4e-3
