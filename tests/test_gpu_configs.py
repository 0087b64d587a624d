"""Parity of the GPU path with the FP64 oracle on two full workloads, against oracle series
stored in tests/golden/ (written by tests/golden/configs.py, which calls only the oracle and
the seeded input generators; the oracle needs about an hour for the first workload):

  * the porous-medium benchmark medium (128^3 random spheres, R = 6, porosity 0.40, seed 1),
    one species, 2e4 FP32 steps -- the full length of the benchmark's MP run;
  * the batched workload's three media (64^3, 128^3, 192^3) x 16 species, 1e3 steps, in one
    group launch; the oracle covers all 16 species of the 64^3 medium and two species of
    each larger one.

Both evaluations of the step (direct with its autotuned variant, and flux) are held to the
bar: Z(t)/Z(0) within 1e-4 absolute and D(t) within 1e-4 relative at every stored time
(every step to 200, then every 25 steps; D(t) sums every Z in between), and total mass
within 1e-5 of the oracle's.
"""
import importlib.util
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
_spec = importlib.util.spec_from_file_location("golden_configs", os.path.join(HERE, "golden", "configs.py"))
configs = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(configs)


@pytest.fixture(scope="module")
def mp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1303_2470_gb300 import build
    build.build()
    from paper_1303_2470_gb300 import mp as m
    return m


def _golden(name):
    path = configs.PATHS[name]
    if not os.path.exists(path):
        pytest.fail(f"{path} is missing: run python tests/golden/configs.py {name}")
    with open(path) as f:
        return json.load(f)


def _check(Z, D, ref, what):
    t = np.asarray(ref["t"])
    Zo, Do = np.asarray(ref["Z"]), np.asarray(ref["D"])
    assert Z.size > t[-1], what
    z_err = np.max(np.abs(Z[t] - Zo)) / abs(Zo[0])
    d_err = np.max(np.abs(D[t] - Do) / np.abs(Do))
    print(f"{what}: Z/Z(0) error {z_err:.3e}, D relative error {d_err:.3e}")
    assert z_err < 1e-4, f"{what}: Z/Z(0) error {z_err:.3e}"
    assert d_err < 1e-4, f"{what}: D relative error {d_err:.3e}"
    return z_err, d_err


@pytest.mark.parametrize("scheme", ["direct", "flux"])
def test_porous128_full_run_matches_oracle(mp, scheme):
    ref = _golden("porous128")
    solid, u, Db, ka, kd, steps = configs.porous128()
    assert ref["steps"] == steps and ref["n_fluid"] == int((solid == 0).sum())
    ud = torch.as_tensor(u).cuda()
    opts = {"scheme": scheme, "autotune": scheme == "direct"}
    stream = torch.cuda.Stream()
    ctx = mp.mp_init(solid, ud, Db, ka, kd, capacity=steps + 30, stream=stream, **opts)
    mp.mp_step(ctx, steps)
    Z, D = mp.mp_vacf(ctx, 0, 0)
    _check(Z, D, ref["series"][0], f"{scheme} ({mp.mp_variant(ctx)})")
    m = mp.mp_mass(ctx, 0)
    want = ref["series"][0]["mass_free"] + ref["series"][0]["mass_ads"]
    assert abs(m[0] + m[1] - want) < 1e-5
    ctx.close()


@pytest.mark.parametrize("scheme", ["direct", "flux"])
def test_batched_group_matches_oracle(mp, scheme):
    ref = _golden("batched")
    meds, steps = configs.batched()
    assert ref["steps"] == steps
    ctxs, streams = [], []
    for solid, u, (Db, ka, kd), _ in meds:
        streams.append(torch.cuda.Stream())
        ctxs.append(mp.mp_init_batch(solid, torch.as_tensor(u).cuda(), Db, ka, kd, capacity=steps + 30,
                                     scheme=scheme, stream=streams[-1]))
    g = mp.mp_group_create(ctxs, graph_steps=64, autotune=True)
    mp.mp_group_step(g, steps)
    variant = mp.mp_group_variant(g)
    g.close()
    for rec in ref["series"]:
        Z, D = mp.mp_vacf(ctxs[rec["medium"]], rec["species"], 0)
        _check(Z, D, rec, f"{scheme} ({variant}) medium {rec['medium']} species {rec['species']}")
        m = mp.mp_mass(ctxs[rec["medium"]], rec["species"])
        assert abs(m[0] + m[1] - (rec["mass_free"] + rec["mass_ads"])) < 1e-5
    for c in ctxs:
        c.close()
