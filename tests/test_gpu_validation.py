"""The paper's validation set (Sec. Validation, Figs. 1-3 and 5) on the GPU, through the C ABI.

Each experiment runs at the paper's sizes (slit L = 100, D_b = 1e-2; fcc unit cell of
lattice parameter 100) and is checked at every sampled time against what is exact for the
lattice (the slit chain, tests/_chains.py; the 3D oracle where it is fast enough) and then,
as the paper does, against the continuum solutions (oracle/continuum.py):
  * Figs. 1-2: wall-normal D(t) for f_a = 0/16/66/95 % and a 5 x 5 (k_a, k_d) grid, FP64;
    relative errors of the slope and origin of the fit of log10 D(t) for D_b t/L^2 in
    [0.5, 1] below the paper's 5 % and 2 %;
  * Fig. 3: Taylor-Aris K along a Poiseuille flow for Pe = 10..120 and the four fractions;
  * Fig. 5: D(t) in the fcc packing for f_a = 0/30/79/97 % (FP32, the production storage).
A summary of the numbers is printed (pytest -s).
"""
import numpy as np
import pytest

import _chains as chains
import oracle
from oracle import continuum as oc
from paper_1303_2470_gb300 import media

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

L, D_b = 100, 0.01
FIG1 = [(0.0, 0.0), (0.1, 1e-2), (0.1, 1e-3), (0.1, 1e-4)]          # f_a = 0, 16, 66, 95 %
GRID = [(a, d) for a in 10.0 ** np.linspace(-3, -1, 5) for d in 10.0 ** np.linspace(-4, -2, 5)]
FIT_TIMES = np.round(np.linspace(0.5, 1.0, 11) * L * L / D_b).astype(np.int64)


@pytest.fixture(scope="module")
def val():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1303_2470_gb300 import build
    build.build()
    from paper_1303_2470_gb300 import validation
    return validation


def test_slit_wall_normal_figs_1_and_2(val):
    pairs = [(0.0, 0.0)] + GRID
    early = np.array([0, 1, 2, 10, 100, 1000, 10_000, 100_000, 300_000])
    times = np.unique(np.concatenate([early, FIT_TIMES]))
    steps = int(FIT_TIMES[-1])
    r = val.slit_wall_normal(pairs, L=L, D_b=D_b, steps=steps, times=times, precision="fp64")
    worst = [0.0, 0.0]
    rows = []
    for s, (ka, kd) in enumerate(pairs):
        ch, pi0 = chains.z_chain(L, np.zeros(L + 2), D_b, ka, kd)
        exact_lattice = chains.zchain_D(ch, pi0, 2, times, confined=True)
        assert np.max(np.abs(r["D"][s] / exact_lattice - 1.0)) < 1e-6, (ka, kd)
        fa = oc.adsorbed_fraction(L, ka, kd)
        total = r["mass"][s, 0] + r["mass"][s, 1]
        assert abs(total - 1.0) < 1e-10 and abs(r["mass"][s, 1] - fa) < 1e-10
        sel = np.isin(times, FIT_TIMES)
        sl, ol = oc.log_fit(times[sel], r["D"][s, sel])
        se, oe = oc.log_fit(times[sel], oc.slit_D(times[sel], L, D_b, ka, kd))
        es, eo = sl / se - 1.0, ol / oe - 1.0
        worst = [max(worst[0], abs(es)), max(worst[1], abs(eo))]
        rows.append((ka, kd, fa, r["D"][s, 0] / D_b, es, eo))
    print("\nslit L=100 D_b=0.01 wall-normal, fit of log10 D(t) for D_b t/L^2 in [0.5, 1] (GPU FP64)")
    print(" k_a       k_d       f_a     D(0)/D_b  slope err  origin err")
    for ka, kd, fa, d0, es, eo in rows:
        print(f" {ka:8.2e}  {kd:8.2e}  {fa:6.3f}  {d0:8.5f}  {es:+9.2e}  {eo:+9.2e}")
    print(f" worst |slope err| {worst[0]:.3e}, worst |origin err| {worst[1]:.3e} (paper: < 5e-2, < 2e-2)")
    assert worst[0] < 0.05 and worst[1] < 0.02


def test_taylor_aris_fig_3(val):
    Pes = [10.0, 30.0, 60.0, 120.0]
    steps = 1_000_000
    times = np.array([0, 1, 10, 1000, 100_000, 500_000, steps])
    r = val.taylor_aris(Pes, FIG1, L=L, D_b=D_b, steps=steps, times=times, precision="fp64")
    print("\nTaylor-Aris K/D_b, slit L=100 D_b=0.01, GPU FP64 after 1e6 steps vs Eq. exact_K")
    print("  Pe     f_a    K_gpu/D_b   K_exact/D_b   gap")
    for i, Pe in enumerate(Pes):
        prof = media.poiseuille_profile(L, r["u_max"][i]).astype(np.float32).astype(np.float64)
        vbar_fluid = prof[1:L + 1].mean()
        for s, (ka, kd) in enumerate(FIG1):
            ch, pi0 = chains.z_chain(L, prof, D_b, ka, kd)
            D_lat = chains.zchain_D(ch, pi0, 0, times)
            assert np.max(np.abs(r["D"][i, s] / D_lat - 1.0)) < 1e-8, (Pe, ka, kd)
            # the stationary drift vbar (mean step of the chain from its Boltzmann weights)
            # removes the ballistic part: K(T) = D(T) - vbar^2 (T + 1/2), within 3e-5 of the
            # chain's asymptotic K after 1e6 steps for all four fractions
            K_inf, vbar = chains.zchain_K(ch, pi0, 0)
            K_gpu = r["D"][i, s, -1] - vbar ** 2 * (steps + 0.5)
            assert abs(K_gpu / K_inf - 1.0) < 1e-4
            y = 0.0 if ka == 0 else ka / (kd * L)
            K_exact = oc.taylor_aris_K(L * vbar_fluid / D_b, y, D_b, L, kd if kd > 0 else 1.0)
            gap = K_gpu / K_exact - 1.0
            print(f" {Pe:5.0f}  {oc.adsorbed_fraction(L, ka, kd):5.3f}  {K_gpu / D_b:10.4f}  {K_exact / D_b:11.4f}"
                  f"  {gap:+.2e}")
            assert abs(gap) < 0.025


def test_fcc_packing_fig_5(val):
    fractions = (0.0, 0.30, 0.79, 0.97)
    a = 100
    R = a * np.sqrt(2.0) / 4.0
    taus = np.array([0.0, 0.05, 0.1, 0.25, 0.5, 0.75, 1.0, 1.5, 2.0])
    times = np.round(taus * R * R / D_b).astype(np.int64)
    r = val.fcc_packing(a=a, fractions=fractions, D_b=D_b, steps=int(times[-1]), times=times, precision="fp32")
    assert abs(r["porosity"] - (1.0 - np.pi / (3.0 * np.sqrt(2.0)))) < 0.005
    solid = media.fcc(a)
    print("\nfcc packing a=100 (R=35.36), D_b=0.01, GPU FP32: D(t)/D_b at D_b t/R^2 =", list(taus))
    for s, (f, (ka, kd)) in enumerate(zip(fractions, r["pairs"])):
        m = r["mass"][s]
        assert abs(m[0] + m[1] - 1.0) < 1e-4
        assert abs(m[1] / (m[0] + m[1]) - f) < 1e-4
        # D(0) = Z(0)/2 at full size, from the oracle's Boltzmann weights and link table
        p = oracle.Problem(solid, None, D_b, ka, kd)
        pi, _ = oracle.equilibrium(p)
        Z0 = oracle.vacf_z0(p, 0, pi)
        assert abs(r["D"][s, 0] / (Z0 / 2.0) - 1.0) < 1e-5
        D = r["D"][s]
        # u = 0: the chain is reversible with positive eigenvalues, so D(t) cannot increase
        assert np.all(np.diff(D) <= 1e-5 * D[:-1]), D
        print(f"  f_a={f:4.2f} (k_a={ka:.3g}, k_d={kd:.3g}): " + " ".join(f"{d / D_b:.4f}" for d in D))


def test_slit_fig_1_fp32_storage(val):
    """Fig. 1's four fractions with FP32 storage (the production precision), against the
    exact lattice. FP32 storage carries a rounding of about 2^-24 of each field value per
    step; a slowly decaying mode accumulates it, and D(t) = Z(0)/2 + sum Z(m) inherits it as
    an absolute error relative to D(0), not to D(t). While D(t) is still a sizeable part of
    D(0) the agreement holds; the wall-normal decay to D_b t/L^2 ~ 1 (D(t) ~ 4e-5 D(0) without
    sorption) is below what FP32 storage resolves, so Fig. 2's fits are done in FP64. The
    deviations are printed; asserted is |D - D_lattice| < 1e-4 D(0) for t <= 1e4 steps."""
    times = np.array([0, 1, 10, 100, 1000, 10_000, 100_000, 300_000, 500_000, 750_000, 1_000_000])
    r = val.slit_wall_normal(FIG1, L=L, D_b=D_b, steps=int(times[-1]), times=times, precision="fp32")
    print("\nslit Fig. 1 cases, FP32 storage: (D - D_lattice)/D(0) at t =", list(times))
    for s, (ka, kd) in enumerate(FIG1):
        ch, pi0 = chains.z_chain(L, np.zeros(L + 2), D_b, ka, kd)
        exact = chains.zchain_D(ch, pi0, 2, times, confined=True)
        dev = (r["D"][s] - exact) / exact[0]
        print(f"  f_a={oc.adsorbed_fraction(L, ka, kd):5.3f}: " + " ".join(f"{d:+.1e}" for d in dev))
        assert np.max(np.abs(dev[times <= 10_000])) < 1e-4


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fcc_cell_matches_oracle(val, precision):
    """Small fcc cell (a = 24, R = a sqrt(2)/4), the four fractions in one batched context,
    300 steps: every species' Z and D against the FP64 oracle."""
    from paper_1303_2470_gb300 import mp
    solid = media.fcc(24)
    pairs = val.fcc_sorption_pairs(solid, (0.0, 0.30, 0.79, 0.97))
    steps = 300
    ctx = mp.mp_init_batch(solid, None, [D_b] * 4, [p[0] for p in pairs], [p[1] for p in pairs],
                           precision=precision, directions="x", capacity=steps + 2)
    mp.mp_step(ctx, steps)
    for s, (ka, kd) in enumerate(pairs):
        Z, D = mp.mp_vacf(ctx, s, 0)
        ref = oracle.run(oracle.Problem(solid, None, D_b, ka, kd), g=0, nsteps=steps)
        if precision == "fp64":
            assert np.max(np.abs(Z - ref.Z)) < 1e-12 * abs(ref.Z[0])
            assert np.max(np.abs(D / ref.D - 1.0)) < 1e-11
        else:
            assert np.max(np.abs(Z - ref.Z)) / abs(ref.Z[0]) < 1e-4
            assert np.max(np.abs(D / ref.D - 1.0)) < 1e-4
    ctx.close()
