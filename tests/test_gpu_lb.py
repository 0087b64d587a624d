"""GPU parity of lb_steady (through the C ABI) against the FP64 oracle LB, and the slit
Poiseuille + sorption pipeline (LB flow feeding the moment propagation) against the oracle.

FP32 populations against the FP64 oracle: velocities within 1e-4 of the largest speed
after a fixed number of steps (the same steps on both sides, tol = 0)."""
import numpy as np
import pytest

import oracle
from paper_1303_2470_gb300 import media

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1303_2470_gb300 import build
    build.build()
    from paper_1303_2470_gb300 import mp as m
    return m


def _u_dev(shape):
    return torch.zeros((3,) + tuple(shape), dtype=torch.float32, device="cuda")


def test_fixed_steps_porous_medium(mp):
    """Ragged 23x26x19 random medium with a sealed pocket, body force in three directions,
    tau = 0.8: u after 400 steps agrees with the oracle's; the pocket stays at rest."""
    solid, _ = media.random_spheres((19, 26, 23), 3, 0.35, seed=5)
    inc, size = oracle.largest_cluster(solid)
    pocket = (solid == 0) & (inc == 0)
    assert pocket.sum() >= 1
    F = (2e-5, -1e-5, 0.5e-5)
    u = _u_dev(solid.shape)
    steps, res, conv = mp.lb_steady(solid, F, u, tau=0.8, tol=0.0, max_steps=400, check_every=50)
    assert steps == 400 and not conv
    uo, so, ro, co = oracle.lb_steady(solid, F, tau=0.8, tol=0.0, max_steps=400, check_every=50)
    ug = u.cpu().numpy().astype(np.float64)
    scale = np.abs(uo).max()
    assert np.max(np.abs(ug - uo)) < 1e-4 * scale
    # the residual is a difference of two FP32 velocities: its error is bounded by a few
    # units in the last place of the largest speed (2^-24 of it), which here is 0.4 % of it
    assert abs(res - ro) < 1e-3 * ro + 4 * 2.0 ** -24 * scale
    assert np.all(ug[:, solid.astype(bool)] == 0.0)
    assert np.all(ug[:, pocket] == 0.0)


def test_density_start_and_output_match_oracle(mp):
    """Started from a given velocity and density (u_init, rho_init) on the same ragged medium,
    300 steps with tau = 0.8: the final u and the density output rho_out agree with the
    oracle's (velocity within 1e-4 of the largest speed, density within 1e-6), solids and the
    sealed pocket keep rho_out 0 and the start density respectively."""
    solid, _ = media.random_spheres((19, 26, 23), 3, 0.35, seed=5)
    fluid = solid == 0
    rng = np.random.default_rng(11)
    u0 = (rng.uniform(-1e-3, 1e-3, (3,) + solid.shape) * fluid).astype(np.float32)
    rho0 = np.where(fluid, 1.0 + rng.uniform(-1e-3, 1e-3, solid.shape), 0.0).astype(np.float32)
    F = (2e-5, -1e-5, 0.5e-5)
    u = _u_dev(solid.shape)
    rho = torch.zeros(solid.shape, dtype=torch.float32, device="cuda")
    steps, _, _ = mp.lb_steady(solid, F, u, tau=0.8, tol=0.0, max_steps=300, check_every=50,
                               u_init=torch.as_tensor(u0).cuda(), rho_init=torch.as_tensor(rho0).cuda(), rho_out=rho)
    assert steps == 300
    uo, _, _, _, ro = oracle.lb_steady(solid, F, tau=0.8, tol=0.0, max_steps=300, check_every=50,
                                       u_init=u0.astype(np.float64), rho_init=rho0.astype(np.float64), with_rho=True)
    ug = u.cpu().numpy().astype(np.float64)
    rg = rho.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(ug - uo)) < 1e-4 * np.abs(uo).max()
    assert np.max(np.abs(rg - ro)) < 1e-6
    assert np.all(rg[~fluid] == 0.0)


def test_classify_matches_oracle(mp):
    """Node classes and the largest fluid cluster are integer work: bit-exact."""
    for shape, R, phi, seed in [((13, 17, 21), 3, 0.5, 1), ((24, 24, 24), 3, 0.30, 7),
                                ((128, 128, 128), 6, 0.40, 1)]:
        solid, _ = media.random_spheres(shape, R, phi, seed)
        for arg in (solid, torch.as_tensor(solid).cuda()):
            cls, (nf, ni, nc) = mp.mp_classify(arg)
            ocls, onf, oni = oracle.classify(solid)
            inc, size = oracle.largest_cluster(solid)
            assert np.array_equal(cls & 3, ocls)
            assert np.array_equal((cls >> 2) & 1, inc)
            assert (nf, ni, nc) == (onf, oni, size)


def test_porous_flow_reaches_the_steady_criterion(mp):
    """128^3 random spheres (R = 6, porosity 0.40, seed 1) at a force giving mean u ~ 0.01:
    with the force on the percolating cluster the residual falls below 1e-7."""
    solid, _ = media.random_spheres((128, 128, 128), 6, 0.40, 1)
    sd = torch.as_tensor(solid).cuda()
    u = _u_dev(solid.shape)
    steps, res, conv = mp.lb_steady(sd, (1.83e-3, 0, 0), u, tol=1e-7, max_steps=100_000, check_every=100)
    assert conv and res < 1e-7
    fl = sd == 0
    assert 0.008 < float(u[0][fl].mean()) < 0.012


def test_rest_stays_at_rest(mp):
    solid, _ = media.random_spheres((16, 16, 16), 3, 0.6, seed=2)
    u = _u_dev(solid.shape)
    steps, res, conv = mp.lb_steady(solid, (0, 0, 0), u, tol=1e-12, max_steps=50, check_every=10)
    assert conv and steps == 10 and res == 0.0
    assert float(u.abs().max()) == 0.0


def test_slit_poiseuille_steady_state(mp):
    """Slit H = 32, tau = 1, F = 8 nu u_max / H^2 (u_max = 0.05): converges below 1e-7 within
    a check period of the oracle, and the profiles agree."""
    H = 32
    F = 8 * (1.0 / 6.0) * 0.05 / H ** 2
    solid = media.slit(16, 16, H)
    u = _u_dev(solid.shape)
    steps, res, conv = mp.lb_steady(solid, (F, 0, 0), u, tol=1e-7, max_steps=200_000, check_every=100)
    uo, so, ro, co = oracle.lb_steady(media.slit(3, 3, H), (F, 0, 0), tol=1e-7, max_steps=200_000,
                                      check_every=100)
    assert conv and co and res < 1e-7
    assert abs(steps - so) <= 200
    ug = u.cpu().numpy()[0, :, 7, 5].astype(np.float64)
    assert np.max(np.abs(ug - uo[0, :, 1, 1])) < 2e-4 * 0.05
    assert np.all(u.cpu().numpy()[0] == u.cpu().numpy()[0, :, :1, :1])   # x,y invariant
    assert abs(ug.max() - 0.05) < 2e-3


def test_not_converged_status_and_warm_start(mp):
    H = 16
    F = 8 * (1.0 / 6.0) * 0.05 / H ** 2
    solid = media.slit(8, 8, H)
    u = _u_dev(solid.shape)
    steps, res, conv = mp.lb_steady(solid, (F, 0, 0), u, tol=1e-7, max_steps=300, check_every=100)
    assert not conv and steps == 300 and res > 1e-7
    with pytest.raises(mp.MPError) as e:
        mp.lb_steady(solid, (F, 0, 0), u, tol=1e-7, max_steps=300, check_every=100,
                     raise_on_unconverged=True)
    assert e.value.code == mp.MP_ENOTCONVERGED
    cold = mp.lb_steady(solid, (F, 0, 0), u, tol=1e-7, max_steps=100_000, check_every=100)
    u2 = _u_dev(solid.shape)
    warm = mp.lb_steady(solid, (F, 0, 0), u2, tol=1e-7, max_steps=100_000, check_every=100, u_init=u)
    assert cold[2] and warm[2] and warm[0] < cold[0]


def test_non_finite_flow_is_not_converged(mp):
    """A start whose density is zero on the fluid blows the velocity up within a few steps
    (the FP32 sum of the populations leaves a density of order 1e-8): the run stops at the
    first check after the velocity is non-finite, long before max_steps, and reports
    MP_ENOTCONVERGED with an infinite residual (a NaN velocity must not pass the residual
    test)."""
    solid, _ = media.random_spheres((16, 16, 16), 3, 0.5, seed=2)
    u = _u_dev(solid.shape)
    rho0 = torch.zeros(solid.shape, dtype=torch.float32, device="cuda")
    steps, res, conv = mp.lb_steady(solid, (1e-5, 0, 0), u, tol=1e-7, max_steps=5000, check_every=10,
                                    rho_init=rho0)
    assert not conv and steps <= 200 and steps % 10 == 0 and np.isinf(res)
    with pytest.raises(mp.MPError) as e:
        mp.lb_steady(solid, (1e-5, 0, 0), u, tol=1e-7, max_steps=5000, check_every=10, rho_init=rho0,
                     raise_on_unconverged=True)
    assert e.value.code == mp.MP_ENOTCONVERGED and "non-finite" in str(e.value)
    # the library stays usable: a plain solve of the same medium converges
    steps, res, conv = mp.lb_steady(solid, (1e-5, 0, 0), u, tol=1e-7, max_steps=100_000, check_every=10)
    assert conv and np.isfinite(res)


@pytest.mark.parametrize("ka,kd", [(0.0, 0.0), (1e-3, 1e-2), (1e-2, 1e-3)])
def test_poiseuille_sorption_pipeline(mp, ka, kd):
    """Slit Poiseuille flow with sorption: 16x16 periodic, H = 32, BGK tau = 1 to 1e-7, MP with
    D_b = 0.02 and 5e4 FP32 steps, the whole pipeline (LB, then MP) on each side."""
    H, steps = 32, 50_000
    F = 8 * (1.0 / 6.0) * 0.05 / H ** 2
    solid = media.slit(16, 16, H)
    # each side solves its own flow: the oracle to 1e-7, then the library for exactly as
    # many steps (the same iteration, so the two flows differ only by FP32 rounding)
    small = media.slit(3, 3, H)
    uo, so, _, co = oracle.lb_steady(small, (F, 0, 0), tol=1e-7, max_steps=200_000, check_every=100)
    assert co
    u = _u_dev(solid.shape)
    n_lb, _, _ = mp.lb_steady(solid, (F, 0, 0), u, tol=0.0, max_steps=so, check_every=100)
    assert n_lb == so
    # lambda/2 = 0.12 < 3 u_max = 0.15: upstream links at the channel centre have p_i < 0;
    # the scheme stays linear and conservative, so they are accepted and counted (R11)
    ctx = mp.mp_init(solid, u, 0.02, ka, kd, capacity=steps + 2, allow_negative=True)
    assert mp.mp_info(ctx)["n_negative_links"] > 0
    mp.mp_step(ctx, steps)
    Z, D = mp.mp_vacf(ctx, 0, 0)
    # the slit is x,y-invariant, so the oracle's 3x3 cross-section has the same Z and D
    ref = oracle.run(oracle.Problem(small, uo, 0.02, ka, kd), g=0, nsteps=steps)
    assert np.max(np.abs(Z - ref.Z)) / abs(ref.Z[0]) < 1e-4
    assert np.max(np.abs(D - ref.D) / np.abs(ref.D)) < 1e-4
    m = mp.mp_mass(ctx, 0)
    assert abs(m[0] + m[1] - 1.0) < 1e-4
    ctx.close()
