"""Binary16 storage of the MP fields (precision "fp16": IEEE binary16 storage, FP32
arithmetic, FP64 reductions), through the C ABI, against the FP64 oracle.

This is a storage variant with no counterpart in the paper; the tests are an error report
with bounds derived from the storage precision. The binary16 unit roundoff is u = 2^-11
(4.9e-4). With stochastic rounding every stored value carries an unbiased error of at most
one spacing per step; Z(t) sums over many nodes, so its error stays a small multiple of u
times |Z(0)| over a few thousand steps. Rounding to nearest is biased wherever a field's
per-step change is below half a spacing (the change is dropped), which is what the report
shows against the stochastic variant.
"""
import numpy as np
import pytest

import oracle
from paper_1303_2470_gb300 import media

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U16 = 2.0 ** -11


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


def _case():
    solid, _ = media.random_spheres((13, 17, 21), 2.5, 0.6, seed=4)      # ragged, 4641 nodes
    u = media.random_flow(solid, 0.02, seed=9).astype(np.float32)
    return solid, u, [0.03, 0.05, 0.08], [0.0, 0.02, 0.05], [0.0, 0.03, 0.01]


def test_fp16_error_report_against_oracle(mp):
    """Three species, moments x and z, 2000 steps: Z/|Z(0)| and D(t) against the oracle for
    both roundings; total mass against 1. Asserted for stochastic rounding: Z within 4u |Z(0)|,
    D within 4u relative, mass within 4u."""
    solid, u, Db, ka, kd = _case()
    steps = 2000
    refs = {(s, g): oracle.run(oracle.Problem(solid, u.astype(np.float64), Db[s], ka[s], kd[s]), g=g, nsteps=steps)
            for s in range(3) for g in (0, 2)}
    print("\nbinary16 storage, 21x17x13 random medium, 2000 steps: max |Z - Z_oracle|/|Z0|, "
          "max |D/D_oracle - 1|, |mass - 1|")
    report = {}
    for rounding in ("stochastic", "nearest"):
        ctx = mp.mp_init_batch(solid, dev32(u), Db, ka, kd, precision="fp16", rounding=rounding,
                               directions="xz", capacity=steps + 2)
        mp.mp_step(ctx, steps)
        for s in range(3):
            m = mp.mp_mass(ctx, s)
            for g in (0, 2):
                Z, D = mp.mp_vacf(ctx, s, g)
                ref = refs[(s, g)]
                ez = np.max(np.abs(Z - ref.Z)) / abs(ref.Z[0])
                ed = np.max(np.abs(D / ref.D - 1.0))
                report[(rounding, s, g)] = (ez, ed, abs(m[0] + m[1] - 1.0))
                print(f"  {rounding:10s} species {s} g={g}: {ez:.2e}  {ed:.2e}  {abs(m[0] + m[1] - 1.0):.2e}")
        ctx.close()
    for s in range(3):
        for g in (0, 2):
            ez, ed, em = report[("stochastic", s, g)]
            assert ez < 4 * U16 and ed < 4 * U16 and em < 4 * U16, (s, g, ez, ed, em)


def test_fp16_is_repeatable_and_field_io_rounds_to_binary16(mp):
    """The stochastic rounding is a hash of (step, element): two runs agree bitwise. Fields
    set through the ABI come back rounded to binary16 (relative 2^-11)."""
    solid, u, Db, ka, kd = _case()
    out = []
    for _ in range(2):
        ctx = mp.mp_init_batch(solid, dev32(u), Db, ka, kd, precision="fp16", capacity=120)
        mp.mp_step(ctx, 100)
        out.append([mp.mp_vacf(ctx, s, 0) for s in range(3)] + [mp.mp_get_field(ctx, 2, 1)])
        ctx.close()
    for a, b in zip(*out):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    ctx = mp.mp_init_batch(solid, dev32(u), Db, ka, kd, precision="fp16", capacity=8)
    rng = np.random.default_rng(3)
    X = (0.5 + 0.5 * rng.random(solid.shape)) * (solid == 0) * 1e-4     # stored values stay normal binary16
    mp.mp_set_field(ctx, 1, 1, X, X)
    G, Ga = mp.mp_get_field(ctx, 1, 1)
    fluid = solid == 0
    assert np.max(np.abs(G[fluid] - X[fluid]) / np.maximum(X[fluid], 1e-30)) <= U16 * 1.0001
    cls, _, _ = oracle.classify(solid)
    itf = cls == 2
    assert np.max(np.abs(Ga[itf] - X[itf]) / np.maximum(X[itf], 1e-30)) <= U16 * 1.0001
    assert np.all(Ga[~itf] == 0.0)
    ctx.close()


def test_fp16_rejections(mp):
    solid, u, _, _, _ = _case()
    with pytest.raises(mp.MPError) as e:
        mp.mp_init(solid, None, 0.05, 0.9, 1e-5, precision="fp16")     # K = 9e4 > 30000
    assert e.value.code == mp.MP_EINVAL
    ctx = mp.mp_init(solid, None, 0.05, 0.01, 0.01, precision="fp16")
    with pytest.raises(mp.MPError) as e:
        mp.mp_group_create([ctx])                                        # groups are FP32 only
    assert e.value.code == mp.MP_EINVAL
    ctx.close()


def test_fp16_against_fp32_on_the_bench_medium(mp):
    """128^3 random spheres (R = 6, porosity 0.40, seed 1), random flow, D_b = 0.05,
    k_a = k_d = 5e-3, 2e4 steps: binary16 storage against FP32 storage (itself within 1e-4 of
    the oracle), reported; asserted D within 10u relative over the run."""
    solid, _ = media.random_spheres((128, 128, 128), 6, 0.40, seed=1)
    u = dev32(media.random_flow(solid, 0.01, seed=3))
    steps = 20_000
    D = {}
    for prec in ("fp32", "fp16"):
        ctx = mp.mp_init(solid, u, 0.05, 5e-3, 5e-3, precision=prec, capacity=steps + 2, allow_negative=True)
        mp.mp_step(ctx, steps)
        D[prec] = mp.mp_vacf(ctx, 0, 0)[1]
        ctx.close()
    rel = np.abs(D["fp16"] / D["fp32"] - 1.0)
    print(f"\nbench medium, 2e4 steps: max |D16/D32 - 1| = {rel.max():.2e}, at t = 2e4: {rel[-1]:.2e}")
    assert rel.max() < 10 * U16
