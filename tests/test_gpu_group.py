"""Grouped stepping (one launch per step for several media and species, CUDA-graph replay,
autotuned block size) against the same contexts stepped one by one."""
import numpy as np
import pytest

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


def _media():
    out = []
    for shape, R, phi, seed, S in [((24, 24, 24), 3, 0.45, 2, 4), ((32, 30, 28), 4, 0.40, 3, 3),
                                   ((40, 36, 44), 4, 0.50, 4, 5)]:
        solid, _ = media.random_spheres(shape, R, phi, seed)
        u = torch.as_tensor(media.random_flow(solid, 0.02, seed=seed + 7).astype(np.float32)).cuda()
        out.append((solid, u, media.species(S, seed=seed + 40)))
    return out


def _contexts(mp, med, cap, directions="x", single=False):
    ctxs = []
    for solid, u, (Db, ka, kd) in med:
        if single:
            Db, ka, kd = Db[:1], ka[:1], kd[:1]
        ctxs.append(mp.mp_init_batch(solid, u, Db, ka, kd, capacity=cap, directions=directions,
                                     allow_negative=True))
    return ctxs


@pytest.mark.parametrize("graph_steps,autotune,single,directions",
                         [(0, False, False, "x"), (64, True, False, "x"), (16, True, True, "x"),
                          (8, False, False, "xz")])
def test_group_equals_separate_contexts(mp, graph_steps, autotune, single, directions):
    med = _media()
    steps = [37, 100, 1, 60]
    cap = sum(steps) + 4
    ref = _contexts(mp, med, cap, directions, single)
    grp = _contexts(mp, med, cap, directions, single)
    g = mp.mp_group_create(grp, graph_steps=graph_steps, autotune=autotune)
    assert mp.mp_group_block_size(g) in (128, 256, 512)
    for n in steps:
        for c in ref:
            mp.mp_step(c, n)
        mp.mp_group_step(g, n)
    torch.cuda.synchronize()
    for c_ref, c_grp in zip(ref, grp):
        info = mp.mp_info(c_ref)
        assert mp.mp_info(c_grp)["t"] == info["t"]
        for s in range(info["n_species"]):
            for f in range(info["n_fields"]):
                a, aa = mp.mp_get_field(c_ref, s, f)
                b, bb = mp.mp_get_field(c_grp, s, f)
                assert np.array_equal(a, b) and np.array_equal(aa, bb)
            for d in ({"x": [0], "xz": [0, 2]}[directions]):
                Za, Da = mp.mp_vacf(c_ref, s, d)
                Zb, Db_ = mp.mp_vacf(c_grp, s, d)
                # identical fields; the Z sums may group the FP32 node terms differently
                # (block size, or the tiled single-species kernel of separate contexts)
                assert np.max(np.abs(Za - Zb)) <= 1e-7 * abs(Za[0])
                assert np.max(np.abs(Da - Db_) / np.abs(Da)) <= 1e-7
    g.close()
    for c in ref + grp:
        c.close()


def test_group_rules(mp):
    med = _media()[:2]
    ctxs = _contexts(mp, med, cap=20)
    g = mp.mp_group_create(ctxs)
    with pytest.raises(mp.MPError) as e:
        mp.mp_step(ctxs[0], 1)                      # grouped contexts step through the group
    assert e.value.code == mp.MP_EINVAL
    with pytest.raises(mp.MPError):
        mp.mp_group_create([ctxs[0]])               # already grouped
    mp.mp_group_step(g, 10)
    with pytest.raises(mp.MPError):
        mp.mp_group_step(g, 10)                     # series full
    g.close()
    mp.mp_step(ctxs[0], 1)                          # free again after the group is gone
    solid, u, _ = med[0]
    c64 = mp.mp_init(solid, None, 0.05, 0.0, 0.0, precision="fp64")  # no flow: no negative links
    with pytest.raises(mp.MPError):
        mp.mp_group_create([c64])                   # groups are FP32
    for c in ctxs + [c64]:
        c.close()
