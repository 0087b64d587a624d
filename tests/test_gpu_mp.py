"""GPU parity of the moment-propagation path (through the C ABI) against the FP64 oracle.

Inputs are seeded and synthetic (tests use the same generators as the benchmark). The bar:
  * FP64 storage: fields, Z(t) and D(t) equal the oracle's to ~1e-12;
  * FP32 storage: Z(t)/Z(0) within 1e-4 absolute and D(t) within 1e-4 relative, fields
    within 1e-5 of the field's largest magnitude per step count tested;
  * integer work (node classes, interface counts) bit-exact.
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


def _z_tol(Zg, Zo):
    return np.max(np.abs(Zg - Zo)) / abs(Zo[0])


def _d_tol(Dg, Do):
    return np.max(np.abs(Dg - Do) / np.maximum(np.abs(Do), 1e-300))


def test_geometry_counts_match_oracle_classes(mp):
    """Node classes are integer work: the fluid and interfacial counts equal the oracle's."""
    for shape, seed in (((13, 17, 21), 1), ((32, 32, 32), 2), ((9, 40, 33), 3)):
        solid, _ = media.random_spheres(shape, 3, 0.5, seed)
        _, nf, ni = oracle.classify(solid)
        ctx = mp.mp_init(solid, None, 0.05, 0.01, 0.01)
        info = mp.mp_info(ctx)
        assert info["n_fluid"] == nf and info["n_interface"] == ni
        assert info["n_nodes"] == solid.size
        # adsorbed partner is nonzero exactly on the oracle's interfacial nodes
        cls, _, _ = oracle.classify(solid)
        _, ads = mp.mp_get_field(ctx, 0, 0)
        assert np.all((ads != 0) == (cls == 2))
        ctx.close()


def test_slit_pure_diffusion_fp64_matches_oracle(mp):
    """8x8 slit, H = 16, u = 0, D_b = 0.05, k_a = k_d = 0.01, density uniform, 1e4 steps,
    FP64 storage: Z, D, mass and all fields agree with the oracle to rounding."""
    H, steps = 16, 10_000
    solid = media.slit(8, 8, H)
    ctx = mp.mp_init(solid, None, 0.05, 0.01, 0.01, precision="fp64", init_density="uniform",
                     capacity=steps + 2)
    mp.mp_step(ctx, steps)
    Z, D = mp.mp_vacf(ctx, 0, 0)
    ref = oracle.run(oracle.Problem(solid, None, 0.05, 0.01, 0.01), g=0, nsteps=steps, init="uniform")
    assert Z.shape == ref.Z.shape
    assert np.max(np.abs(Z - ref.Z)) < 1e-14
    assert np.max(np.abs(D - ref.D)) < 1e-12
    m = mp.mp_mass(ctx, 0)
    assert abs(m[0] + m[1] - 1.0) < 1e-12
    assert abs(m[1] / m[2] - 1.0) < 1e-10          # Gamma/rho -> K = 1
    P, Pa = mp.mp_get_field(ctx, 0, 0)
    assert np.max(np.abs(P - ref.P)) < 1e-15 and np.max(np.abs(Pa - ref.Pa)) < 1e-15
    G, Ga = mp.mp_get_field(ctx, 0, 1)
    assert np.max(np.abs(G - ref.Pg)) < 1e-15 and np.max(np.abs(Ga - ref.Pga)) < 1e-15
    # lateral plateau, lattice closed form
    assert np.max(np.abs(D - 0.05 * (H - 1.0 / 3.0) / (H + 2.0))) < 1e-12
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_random_medium_flow_sorption_all_directions(mp, precision):
    """Ragged 21x17x13 random medium (N not a multiple of 32), random flow, three species,
    x/y/z moments: every species, direction, series and field matches the oracle."""
    solid, _ = media.random_spheres((13, 17, 21), 2.5, 0.6, seed=4)
    u = media.random_flow(solid, 0.03, seed=9).astype(np.float32)
    Db, ka, kd = [0.03, 0.05, 0.08], [0.0, 0.02, 0.05], [0.0, 0.03, 0.01]
    steps = 300
    ctx = mp.mp_init_batch(solid, dev32(u), Db, ka, kd, precision=precision, directions="xyz",
                           capacity=steps + 2)
    mp.mp_step(ctx, steps)
    for s in range(3):
        for g in range(3):
            Z, D = mp.mp_vacf(ctx, s, g)
            ref = oracle.run(oracle.Problem(solid, u.astype(np.float64), Db[s], ka[s], kd[s]), g=g,
                             nsteps=steps)
            if precision == "fp64":
                assert np.max(np.abs(Z - ref.Z)) < 1e-14 * abs(ref.Z[0]) * 100
                assert _d_tol(D, ref.D) < 1e-11
                G, Ga = mp.mp_get_field(ctx, s, 1 + g)
                assert np.max(np.abs(G - ref.Pg)) < 1e-13 * np.abs(ref.Pg).max()
                assert np.max(np.abs(Ga - ref.Pga)) < 1e-13 * max(np.abs(ref.Pga).max(), 1e-300)
            else:
                assert _z_tol(Z, ref.Z) < 1e-4
                assert _d_tol(D, ref.D) < 1e-4
                G, _ = mp.mp_get_field(ctx, s, 1 + g)
                assert np.max(np.abs(G - ref.Pg)) < 1e-5 * np.abs(ref.Pg).max()
        P, Pa = mp.mp_get_field(ctx, s, 0)
        tol = 1e-13 if precision == "fp64" else 1e-5
        assert np.max(np.abs(P - ref.P)) < tol * ref.P.max()
        assert np.max(np.abs(Pa - ref.Pa)) < tol * max(ref.Pa.max(), 1e-300)
    ctx.close()


def test_batch_equals_single_species_runs(mp):
    """Species in one batched launch give bitwise the same fields as one species per
    context; Z and D agree to the rounding of the FP32 mean-step sum (the batched path forms
    u*_g as sum w q c + lambda/2 sum w c, the single path sums p c link by link)."""
    solid, _ = media.random_spheres((24, 20, 36), 3, 0.55, seed=8)
    u = dev32(media.random_flow(solid, 0.02, seed=2))
    Db, ka, kd = media.species(5, seed=12)
    ctx = mp.mp_init_batch(solid, u, Db, ka, kd, capacity=102, allow_negative=True)
    mp.mp_step(ctx, 100)
    for s in range(5):
        one = mp.mp_init(solid, u, Db[s], ka[s], kd[s], capacity=102, allow_negative=True)
        mp.mp_step(one, 100)
        for f in range(2):
            a, aa = mp.mp_get_field(ctx, s, f)
            b, bb = mp.mp_get_field(one, 0, f)
            assert np.array_equal(a, b) and np.array_equal(aa, bb)
        Zb, Db_ = mp.mp_vacf(ctx, s, 0)
        Z1, D1 = mp.mp_vacf(one, 0, 0)
        assert np.max(np.abs(Zb - Z1)) <= 1e-6 * abs(Z1[0])
        assert np.max(np.abs(Db_ - D1) / np.abs(D1)) <= 1e-6
        one.close()
    ctx.close()


def test_repeatable_bitwise(mp):
    solid, _ = media.random_spheres((40, 40, 40), 4, 0.45, seed=6)
    u = dev32(media.random_flow(solid, 0.01, seed=1))
    out = []
    for _ in range(2):
        ctx = mp.mp_init(solid, u, 0.05, 5e-3, 5e-3, capacity=60)
        mp.mp_step(ctx, 50)
        out.append(mp.mp_vacf(ctx, 0, 0))
        ctx.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_bulk_box_without_interface(mp):
    """No solid node at all (no interfacial node, empty adsorbed arrays): D(t) = D_b."""
    solid = media.bulk(33, 5, 7)
    ctx = mp.mp_init(solid, None, 0.07, 0.01, 0.02, precision="fp64", capacity=30)
    mp.mp_step(ctx, 25)
    Z, D = mp.mp_vacf(ctx, 0, 0)
    assert np.max(np.abs(D - 0.07)) < 1e-15 and np.max(np.abs(Z[1:])) < 1e-17
    assert mp.mp_info(ctx)["n_interface"] == 0
    ctx.close()


def test_single_step_field_parity_at_full_size(mp):
    """128^3 random spheres (R = 6, porosity 0.40, seed 1): one step from an arbitrary
    seeded state, every field value against the oracle's step (FP32 storage)."""
    solid, _ = media.random_spheres((128, 128, 128), 6, 0.40, seed=1)
    u = media.random_flow(solid, 0.01, seed=3).astype(np.float32)
    ctx = mp.mp_init(solid, dev32(u), 0.05, 5e-3, 5e-3)
    rng = np.random.default_rng(5)
    X = rng.random(solid.shape) * (solid == 0)
    cls, _, _ = oracle.classify(solid)
    Xa = rng.random(solid.shape) * (cls == 2)
    X32, Xa32 = X.astype(np.float32).astype(np.float64), Xa.astype(np.float32).astype(np.float64)
    mp.mp_set_field(ctx, 0, 1, X32, Xa32)
    mp.mp_step(ctx, 1)
    G, Ga = mp.mp_get_field(ctx, 0, 1)
    Xn, Xan = oracle.propagate(oracle.Problem(solid, u.astype(np.float64), 0.05, 5e-3, 5e-3), X32, Xa32)
    assert np.max(np.abs(G - Xn)) < 2e-6 * np.abs(Xn).max()
    assert np.max(np.abs(Ga - Xan)) < 2e-6 * np.abs(Xan).max()
    ctx.close()


def test_errors_are_status_codes(mp):
    solid = media.slit(4, 4, 6)
    with pytest.raises(mp.MPError) as e:
        mp.mp_init(solid, None, 0.3, 0.0, 0.0)           # D_b out of range
    assert e.value.code == mp.MP_EINVAL
    with pytest.raises(mp.MPError) as e:
        mp.mp_init(solid, None, 0.05, 0.1, 0.0)           # no equilibrium
    assert e.value.code == mp.MP_EINVAL
    with pytest.raises(mp.MPError) as e:
        mp.mp_init(np.ones((4, 4, 4), np.uint8), None, 0.05, 0.0, 0.0)   # no fluid
    assert e.value.code == mp.MP_EINVAL
    u = np.zeros((3,) + solid.shape, np.float32)
    u[0, 1:-1] = 0.3                                      # 3 u > lambda/2 on upstream links
    with pytest.raises(mp.MPError) as e:
        mp.mp_init(solid, dev32(u), 0.02, 0.0, 0.0)
    assert e.value.code == mp.MP_ENEGPROB
    ctx = mp.mp_init(solid, dev32(u), 0.02, 0.0, 0.0, allow_negative=True)
    assert mp.mp_info(ctx)["n_negative_links"] > 0
    ctx.close()
    ctx = mp.mp_init(solid, None, 0.05, 0.0, 0.0, capacity=10)
    mp.mp_step(ctx, 8)
    with pytest.raises(mp.MPError) as e:
        mp.mp_step(ctx, 2)                                 # series full
    assert e.value.code == mp.MP_EINVAL
    ctx.close()


def test_graph_replay_equals_plain_launches(mp):
    """A context on its own stream replays long runs from a CUDA graph; the fields and the
    Z/D series equal those of plain launches on the default stream bitwise, including a
    run that starts from the other buffer (after an odd number of steps)."""
    solid, _ = media.random_spheres((20, 24, 28), 3, 0.5, seed=14)
    u = dev32(media.random_flow(solid, 0.02, seed=6))
    st = torch.cuda.Stream()
    out = []
    for stream in (None, st):
        ctx = mp.mp_init_batch(solid, u, [0.04, 0.06], [0.01, 0.0], [0.02, 0.0], capacity=700, stream=stream,
                               directions="xz")
        for n in (3, 300, 129, 200):          # odd first run: the graph for the other buffer
            mp.mp_step(ctx, n)
        res = [mp.mp_get_field(ctx, s, f) for s in range(2) for f in range(3)]
        res += [mp.mp_vacf(ctx, s, g) for s in range(2) for g in (0, 2)]
        out.append(res)
        ctx.close()
    for a, b in zip(*out):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("precision", ["fp32", "fp64", "fp16"])
def test_maximum_species_count_all_directions(mp, precision):
    """MP_MAX_SPECIES = 32 species with x, y and z moments in one context (the largest number
    of chunk passes of the multi-species step) on a ragged 15x11x17 medium with flow, 120
    steps: sampled species against the oracle (FP64 1e-11; FP32 and binary16 storage with
    stochastic rounding 1e-4 and 2e-3 in D); 33 species are rejected."""
    solid, _ = media.random_spheres((17, 11, 15), 2.5, 0.55, seed=21)
    u = media.random_flow(solid, 0.02, seed=22).astype(np.float32)
    Db, ka, kd = media.species(32, seed=23)
    steps = 120
    ctx = mp.mp_init_batch(solid, dev32(u), Db, ka, kd, precision=precision, directions="xyz", capacity=steps + 2,
                           allow_negative=True)
    mp.mp_step(ctx, steps)
    for s in (0, 13, 31):
        for g in range(3):
            Z, D = mp.mp_vacf(ctx, s, g)
            ref = oracle.run(oracle.Problem(solid, u.astype(np.float64), Db[s], ka[s], kd[s]), g=g, nsteps=steps)
            if precision == "fp64":
                assert _d_tol(D, ref.D) < 1e-11
            else:
                assert _z_tol(Z, ref.Z) < (1e-4 if precision == "fp32" else 2e-3)
                assert _d_tol(D, ref.D) < (1e-4 if precision == "fp32" else 2e-3)
    ctx.close()
    Db33, ka33, kd33 = media.species(33, seed=24)
    with pytest.raises(mp.MPError) as e:
        mp.mp_init_batch(solid, dev32(u), Db33, ka33, kd33)
    assert e.value.code == mp.MP_EINVAL
