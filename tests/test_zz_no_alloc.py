"""The allocation-free step (mp_step_noalloc) against the ordinary path, through the C ABI.

mp_step_noalloc is for callers that cannot let a library allocate device memory -- for
instance a solver embedded in a host application that owns every device allocation, or code
that must not trigger the device-wide synchronisation of cudaMalloc/cudaFree. It keeps its
reduction scratch in a fixed device array instead. Here two calls in a row, each fed the
previous call's output, must reproduce two mp_step calls of a context started from the same
field, within the FP32 parity tolerance of the other GPU tests. The file is named to be
collected last, and passes alone in a fresh process as well as after the other tests.
"""
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


def test_noalloc_step_matches_mp_step_on_two_calls(mp):
    solid, _ = media.random_spheres((28, 36, 40), 3, 0.5, seed=31)   # N = 40320, ragged
    u = media.random_flow(solid, 0.03, seed=4).astype(np.float32)
    D_b, k_a, k_d = 0.04, 0.02, 0.03
    rng = np.random.default_rng(8)
    fluid = solid == 0
    X = (rng.random(solid.shape) * fluid).astype(np.float32)
    Xa = (rng.random(solid.shape) * fluid).astype(np.float32)

    dev = torch.device("cuda")
    solid_d = torch.as_tensor(solid).to(dev)
    u_d = torch.as_tensor(u).to(dev)
    x_in, xa_in = torch.as_tensor(X).to(dev), torch.as_tensor(Xa).to(dev)
    x_out, xa_out = torch.empty_like(x_in), torch.empty_like(xa_in)
    z = torch.zeros(1, dtype=torch.float64, device=dev)

    ctx = mp.mp_init(solid_d, u_d, D_b, k_a, k_d, capacity=8)
    mp.mp_set_field(ctx, 0, 1, X.astype(np.float64), Xa.astype(np.float64))
    for call in range(2):
        mp.mp_step(ctx, 1)
        G, Ga = mp.mp_get_field(ctx, 0, 1)
        Z, _ = mp.mp_vacf(ctx, 0, 0)
        mp.mp_step_noalloc(solid_d, u_d, D_b, k_a, k_d, 0, x_in, xa_in, x_out, xa_out, z)
        torch.cuda.synchronize()
        got = x_out.cpu().numpy().astype(np.float64)
        got_a = xa_out.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got - G)) <= 1e-6 * np.abs(G).max(), f"call {call}: field"
        assert np.max(np.abs(got_a - Ga)) <= 1e-6 * np.abs(Ga).max(), f"call {call}: adsorbed"
        assert abs(float(z.item()) - Z[-1]) <= 1e-6 * abs(Z[-1]), f"call {call}: sum"
        x_in, x_out = x_out, x_in
        xa_in, xa_out = xa_out, xa_in
    ctx.close()


def test_noalloc_rejects_oversized_lattices_and_aliasing(mp):
    dev = torch.device("cuda")
    small = torch.zeros((4, 4, 4), dtype=torch.uint8, device=dev)
    a = torch.zeros((4, 4, 4), dtype=torch.float32, device=dev)
    b, c, d = torch.zeros_like(a), torch.zeros_like(a), torch.zeros_like(a)
    z = torch.zeros(1, dtype=torch.float64, device=dev)
    with pytest.raises(mp.MPError) as e:
        mp.mp_step_noalloc(small, None, 0.05, 0.0, 0.0, 0, a, b, a, d, z)      # X_out aliases X
    assert e.value.code == mp.MP_EINVAL

    class Big:  # shape beyond the scratch limit; nothing is dereferenced before the check
        shape = (129, 128, 128)

        def data_ptr(self):
            return int(a.data_ptr())
    with pytest.raises(mp.MPError) as e:
        mp.mp_step_noalloc(Big(), None, 0.05, 0.0, 0.0, 0, a, b, c, d, z)
    assert e.value.code == mp.MP_EINVAL and "exceed" in str(e.value)
