"""GPU parity of the direct evaluation of the step (MP_SCHEME_DIRECT, the paper's form
X' = sum_i p_i X(r - c_i) + stay X) against the FP64 oracle, through the C ABI, for every
kernel variant; the variants against each other; direct groups; the bounded device-wide
barrier of the persistent variant.

The bar is the one of the FP32 flux path: Z(t)/Z(0) within 1e-4 absolute, D(t) within 1e-4
relative, fields within 1e-5 of their largest magnitude.
"""
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


def dev32(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _z_err(Zg, Zo):
    return np.max(np.abs(Zg - Zo)) / abs(Zo[0])


def _d_err(Dg, Do):
    return np.max(np.abs(Dg - Do) / np.maximum(np.abs(Do), 1e-300))


def _variants(mp):
    R, P, B1, B5 = mp.MP_VARIANT_RECOMPUTE, mp.MP_VARIANT_PERSISTENT, mp.MP_VARIANT_BLOCK128, mp.MP_VARIANT_BLOCK512
    T = mp.MP_VARIANT_TILED
    return [0, R, P, R | P, B1, P | B5, R | P | B1, T, T | R, T | P, T | R | P]


@pytest.mark.parametrize("species", [1, 3, 9])
@pytest.mark.parametrize("dirs", ["x", "xyz"])
def test_direct_matches_oracle_every_variant(mp, species, dirs):
    """Ragged 21x17x13 random medium with flow and sorption, 300 steps: every variant's Z, D
    and fields match the oracle; all variants give identical fields, and series equal up to
    the order of their FP64 partial sums (tiled variants with several species: up to the
    grouping of their FP32 warp sums, which covers other nodes)."""
    solid, _ = media.random_spheres((13, 17, 21), 2.5, 0.6, seed=4)
    u = media.drift_flow(solid, 0.01, 0.02, seed=9).astype(np.float32)
    Db, ka, kd = media.species(species, seed=40 + species, D_b=(0.03, 0.1), k=(1e-3, 5e-2))
    steps = 300
    refs = {(s, g): oracle.run(oracle.Problem(solid, u.astype(np.float64), Db[s], ka[s], kd[s]), g=g, nsteps=steps)
            for s in range(species) for g in range(len(dirs))}
    first = None
    for var in _variants(mp):
        ctx = mp.mp_init_batch(solid, dev32(u), Db, ka, kd, directions=dirs, capacity=steps + 2, scheme="direct",
                               variant=var)
        assert mp.mp_variant(ctx).split(",")[0] == ("persistent" if var & mp.MP_VARIANT_PERSISTENT else "per-step")
        mp.mp_step(ctx, steps)
        got = []
        for s in range(species):
            for g in range(len(dirs)):
                Z, D = mp.mp_vacf(ctx, s, g)
                ref = refs[(s, g)]
                assert _z_err(Z, ref.Z) < 1e-4, (var, s, g)
                assert _d_err(D, ref.D) < 1e-4, (var, s, g)
                G, Ga = mp.mp_get_field(ctx, s, 1 + g)
                assert np.max(np.abs(G - ref.Pg)) < 1e-5 * np.abs(ref.Pg).max()
                got += [("series", Z), ("series", D), ("field", G), ("field", Ga)]
            P, Pa = mp.mp_get_field(ctx, s, 0)
            ref = refs[(s, 0)]
            assert np.max(np.abs(P - ref.P)) < 1e-5 * ref.P.max()
            assert np.max(np.abs(Pa - ref.Pa)) < 1e-5 * max(ref.Pa.max(), 1e-300)
            got += [("field", P), ("field", Pa)]
        if first is None:
            first = got
        else:
            for (kind, a), (_, b) in zip(first, got):
                if kind == "field":
                    assert np.array_equal(a, b), var
                else:
                    tol = 1e-6 if (var & mp.MP_VARIANT_TILED and species > 1) else 1e-12
                    assert np.max(np.abs(a - b)) <= tol * np.abs(b).max(), var
        ctx.close()


def test_direct_and_flux_agree_and_conserve_mass(mp):
    """One species on a 40x36x28 medium with flow, 2000 steps: the direct and the flux
    evaluations give the same fields to FP32 rounding, and the direct form keeps the total
    mass to 1e-6 (its stay fraction is rounded once per node)."""
    solid, _ = media.random_spheres((28, 36, 40), 3, 0.45, seed=12)
    u = dev32(media.drift_flow(solid, 0.01, 0.01, seed=3))
    ctxs = [mp.mp_init(solid, u, 0.05, 5e-3, 5e-3, capacity=2002, scheme=sc) for sc in ("flux", "direct")]
    for c in ctxs:
        mp.mp_step(c, 2000)
    for f in range(2):
        a, aa = mp.mp_get_field(ctxs[0], 0, f)
        b, bb = mp.mp_get_field(ctxs[1], 0, f)
        assert np.max(np.abs(a - b)) < 1e-5 * np.abs(a).max()
        assert np.max(np.abs(aa - bb)) < 1e-5 * np.abs(aa).max()
    m = mp.mp_mass(ctxs[1], 0)
    assert abs(m[0] + m[1] - 1.0) < 1e-6
    Zf, Df = mp.mp_vacf(ctxs[0], 0, 0)
    Zd, Dd = mp.mp_vacf(ctxs[1], 0, 0)
    assert _z_err(Zd, Zf) < 1e-5 and _d_err(Dd, Df) < 1e-5
    for c in ctxs:
        c.close()


def test_autotune_keeps_state_and_matches_oracle(mp):
    """Autotuning at mp_init times every variant on the initial state and restores it: the
    series and fields afterwards equal an untuned context's, and the run matches the oracle."""
    solid, _ = media.random_spheres((24, 20, 36), 3, 0.55, seed=8)
    u = media.drift_flow(solid, 0.005, 0.01, seed=2).astype(np.float32)
    Db, ka, kd = media.species(5, seed=12, D_b=(0.03, 0.1))
    steps = 200
    tuned = mp.mp_init_batch(solid, dev32(u), Db, ka, kd, capacity=steps + 30, scheme="direct", autotune=True)
    plain = mp.mp_init_batch(solid, dev32(u), Db, ka, kd, capacity=steps + 30, scheme="direct")
    assert mp.mp_info(tuned)["t"] == 1
    for s in range(5):
        assert np.array_equal(mp.mp_get_field(tuned, s, 0)[0], mp.mp_get_field(plain, s, 0)[0])
        assert np.array_equal(mp.mp_vacf(tuned, s, 0)[0], mp.mp_vacf(plain, s, 0)[0])
    mp.mp_step(tuned, steps)
    for s in range(5):
        Z, D = mp.mp_vacf(tuned, s, 0)
        ref = oracle.run(oracle.Problem(solid, u.astype(np.float64), Db[s], ka[s], kd[s]), g=0, nsteps=steps)
        assert Z.size == steps + 2
        assert _z_err(Z, ref.Z) < 1e-4 and _d_err(D, ref.D) < 1e-4
    tuned.close()
    plain.close()


@pytest.mark.parametrize("autotune,variant", [(False, 0), (True, 0), (False, 16 | 2), (False, 16)])
def test_direct_group_of_uneven_media(mp, autotune, variant):
    """Three media of different sizes, 4, 1 and 6 species, advanced by one launch per step
    (or one persistent launch; autotuned, or the tiled variant, whose launch also steps the
    one-species medium untiled): identical fields to each context stepped on its own, and
    every species matches the oracle."""
    shapes = [(16, 18, 20), (24, 24, 24), (20, 12, 28)]
    nsp = [4, 1, 6]
    steps = 150
    ctxs, inputs = [], []
    for j, (shape, S) in enumerate(zip(shapes, nsp)):
        solid, _ = media.random_spheres(shape, [2, 3, 4], 0.55, seed=60 + j)
        u = media.drift_flow(solid, 0.005, 0.004, seed=70 + j).astype(np.float32)
        sp = media.species(S, seed=80 + j)
        inputs.append((solid, u, sp))
        ctxs.append(mp.mp_init_batch(solid, dev32(u), *sp, capacity=steps + 40, scheme="direct"))
    g = mp.mp_group_create(ctxs, autotune=autotune, variant=variant)
    assert mp.mp_group_variant(g) != "flux"
    if variant & mp.MP_VARIANT_TILED:
        assert "tiled" in mp.mp_group_variant(g)
    mp.mp_group_step(g, steps)
    g.close()
    for c, (solid, u, (Db, ka, kd)) in zip(ctxs, inputs):
        alone = mp.mp_init_batch(solid, dev32(u), Db, ka, kd, capacity=steps + 40, scheme="direct")
        mp.mp_step(alone, steps)
        for s in range(len(Db)):
            for f in range(2):
                a, aa = mp.mp_get_field(c, s, f)
                b, bb = mp.mp_get_field(alone, s, f)
                assert np.array_equal(a, b) and np.array_equal(aa, bb)
            Z, D = mp.mp_vacf(c, s, 0)
            ref = oracle.run(oracle.Problem(solid, u.astype(np.float64), Db[s], ka[s], kd[s]), g=0, nsteps=steps)
            assert _z_err(Z, ref.Z) < 1e-4 and _d_err(D, ref.D) < 1e-4
        # after the group is freed the context steps on its own again, continuing its run
        mp.mp_step(c, 10)
        mp.mp_step(alone, 10)
        assert np.array_equal(mp.mp_get_field(c, 0, 1)[0], mp.mp_get_field(alone, 0, 1)[0])
        alone.close()
        c.close()


def test_grid_barrier_wait_gives_up_and_device_stays_usable(mp):
    """The persistent step's device-wide barrier: reachable barriers pass; a barrier that
    waits for an arrival that never comes gives up after its time limit with MP_ETIMEOUT,
    and the device runs ordinary work afterwards."""
    mp.mp_grid_wait_selftest(64, 200, False, 1_000_000_000)
    with pytest.raises(mp.MPError) as e:
        mp.mp_grid_wait_selftest(64, 3, True, 2_000_000)
    assert e.value.code == mp.MP_ETIMEOUT
    mp.mp_grid_wait_selftest(64, 10, False, 1_000_000_000)
    solid, _ = media.random_spheres((12, 12, 12), 2, 0.6, seed=1)
    ctx = mp.mp_init(solid, None, 0.05, 0.0, 0.0, capacity=20, scheme="direct", variant=mp.MP_VARIANT_PERSISTENT)
    mp.mp_step(ctx, 10)
    Z, D = mp.mp_vacf(ctx, 0, 0)
    assert Z.size == 12 and np.all(np.isfinite(D))
    ctx.close()


def test_direct_rejects_other_precisions(mp):
    solid = media.slit(4, 4, 6)
    for prec in ("fp64", "fp16"):
        with pytest.raises(mp.MPError) as e:
            mp.mp_init(solid, None, 0.05, 0.0, 0.0, precision=prec, scheme="direct")
        assert e.value.code == mp.MP_EINVAL


def test_sharded_units_through_the_library_match_oracle(mp):
    """The split of (medium, species) units (here on one rank) run through the library:
    each medium's share becomes one context; every unit's series matches the oracle."""
    from paper_1303_2470_gb300 import shard
    meds = []
    for j, shape in enumerate(((9, 10, 11), (8, 12, 7))):
        solid, _ = media.random_spheres(shape, 2, 0.6, seed=20 + j)
        u = media.drift_flow(solid, 0.005, 0.004, seed=30 + j).astype(np.float32)
        meds.append((solid, u, media.species(3, seed=40 + j, D_b=(0.03, 0.1))))
    dev_media = [(s, dev32(u), sp) for s, u, sp in meds]
    units = [(m, s) for m in range(2) for s in (0, 2)]
    got = shard.run_sharded(dev_media, units, 60, shard.mp_medium_runner(mp, scheme="direct"))
    assert sorted(got) == sorted(units)
    for (m, s), (Z, D) in got.items():
        solid, u, (Db, ka, kd) = meds[m]
        ref = oracle.run(oracle.Problem(solid, u.astype(np.float64), Db[s], ka[s], kd[s]), g=0, nsteps=60)
        assert _z_err(Z, ref.Z) < 1e-4 and _d_err(D, ref.D) < 1e-4


def test_field_io_of_fluid_list_storage(mp):
    """Several species in the direct scheme keep their fields over the fluid list only:
    mp_set_field then mp_get_field returns the dense input on fluid nodes and zero on solids,
    and a step from the set state equals the flux scheme's (dense storage) to FP32 rounding,
    with the total mass kept."""
    solid, _ = media.random_spheres((14, 15, 17), 2.5, 0.55, seed=21)
    u = dev32(media.drift_flow(solid, 0.01, 0.01, seed=22))
    Db, ka, kd = media.species(3, seed=23, D_b=(0.03, 0.1))
    rng = np.random.default_rng(24)
    X = rng.random(solid.shape) * (solid == 0)
    Xa = rng.random(solid.shape) * (solid == 0)
    ctxs = [mp.mp_init_batch(solid, u, Db, ka, kd, capacity=20, scheme=sc) for sc in ("direct", "flux")]
    for c in ctxs:
        mp.mp_set_field(c, 2, 0, X, Xa)
    G, Ga = mp.mp_get_field(ctxs[0], 2, 0)
    assert np.array_equal(G, X.astype(np.float32).astype(np.float64))
    assert np.all(G[solid != 0] == 0)
    ifc = Ga != 0
    assert np.array_equal(Ga[ifc], Xa.astype(np.float32).astype(np.float64)[ifc])
    m0 = mp.mp_mass(ctxs[0], 2)
    for c in ctxs:
        mp.mp_step(c, 3)
    for f in range(2):
        a, aa = mp.mp_get_field(ctxs[0], 2, f)
        b, bb = mp.mp_get_field(ctxs[1], 2, f)
        assert np.max(np.abs(a - b)) <= 1e-5 * np.abs(b).max()
        assert np.max(np.abs(aa - bb)) <= 1e-5 * max(np.abs(bb).max(), 1e-30)
    m1 = mp.mp_mass(ctxs[0], 2)
    assert abs((m1[0] + m1[1]) - (m0[0] + m0[1])) <= 1e-6 * (m0[0] + m0[1])
    for c in ctxs:
        c.close()
