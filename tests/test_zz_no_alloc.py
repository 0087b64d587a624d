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


@pytest.mark.parametrize("direction", [-1, 0, 1, 2])
@pytest.mark.parametrize("flow", [True, False])
def test_noalloc_step_matches_mp_step_on_two_calls(mp, direction, flow):
    """direction g = 0, 1, 2 weights the sum by u*_g and is compared with mp_vacf of that
    direction (the field is then the propagated g moment); direction -1 is the plain sum of
    the new field, compared with the FP64 sum of the field that mp_step produced."""
    solid, _ = media.random_spheres((28, 36, 40), 3, 0.5, seed=31)   # N = 40320, ragged
    u = media.random_flow(solid, 0.03, seed=4).astype(np.float32) if flow else None
    D_b, k_a, k_d = 0.04, 0.02, 0.03
    rng = np.random.default_rng(8 + direction)
    fluid = solid == 0
    X = (rng.random(solid.shape) * fluid).astype(np.float32)
    Xa = (rng.random(solid.shape) * fluid).astype(np.float32)
    g = max(direction, 0)

    dev = torch.device("cuda")
    solid_d = torch.as_tensor(solid).to(dev)
    u_d = torch.as_tensor(u).to(dev) if flow else None
    x_in, xa_in = torch.as_tensor(X).to(dev), torch.as_tensor(Xa).to(dev)
    x_out, xa_out = torch.empty_like(x_in), torch.empty_like(xa_in)
    z = torch.zeros(1, dtype=torch.float64, device=dev)

    ctx = mp.mp_init(solid_d, u_d, D_b, k_a, k_d, capacity=8, directions="xyz")
    mp.mp_set_field(ctx, 0, 1 + g, X.astype(np.float64), Xa.astype(np.float64))
    for call in range(2):
        mp.mp_step(ctx, 1)
        G, Ga = mp.mp_get_field(ctx, 0, 1 + g)
        want = float(G.sum()) if direction < 0 else mp.mp_vacf(ctx, 0, g)[0][-1]
        mp.mp_step_noalloc(solid_d, u_d, D_b, k_a, k_d, direction, x_in, xa_in, x_out, xa_out, z)
        torch.cuda.synchronize()
        got = x_out.cpu().numpy().astype(np.float64)
        got_a = xa_out.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got - G)) <= 1e-6 * np.abs(G).max(), f"call {call}: field"
        assert np.max(np.abs(got_a - Ga)) <= 1e-6 * np.abs(Ga).max(), f"call {call}: adsorbed"
        # FP32 products summed in different orders: bounded by the magnitude of the terms
        # (|u*_g| < 0.1 here), not only of the possibly cancelling total
        assert abs(float(z.item()) - want) <= 1e-6 * abs(want) + 1e-8 * np.abs(G).sum(), f"call {call}: sum"
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

    class Big:  # a uint8 mask beyond the scratch limit; nothing is dereferenced before the check
        shape = (129, 128, 128)
        is_cuda = True
        dtype = torch.uint8
        device = a.device

        def is_contiguous(self):
            return True

        def data_ptr(self):
            return int(a.data_ptr())
    n_big = 129 * 128 * 128
    big = [torch.zeros(n_big, dtype=torch.float32, device=dev) for _ in range(4)]
    with pytest.raises(mp.MPError) as e:
        mp.mp_step_noalloc(Big(), None, 0.05, 0.0, 0.0, 0, *big, z)
    assert e.value.code == mp.MP_EINVAL and "exceed" in str(e.value)

    # an output that is an offset view into an input overlaps it without sharing its base
    buf = torch.zeros(2 * 64 + 16, dtype=torch.float32, device=dev)
    x_view, out_view = buf[:64].view(4, 4, 4), buf[8:72].view(4, 4, 4)
    with pytest.raises(mp.MPError) as e:
        mp.mp_step_noalloc(small, None, 0.05, 0.0, 0.0, 0, x_view, b, out_view, d, z)
    assert e.value.code == mp.MP_EINVAL and "overlap" in str(e.value)


def test_noalloc_binding_refuses_mismatched_buffers(mp):
    dev = torch.device("cuda")
    small = torch.zeros((4, 4, 4), dtype=torch.uint8, device=dev)
    a = torch.zeros((4, 4, 4), dtype=torch.float32, device=dev)
    b, c, d = torch.zeros_like(a), torch.zeros_like(a), torch.zeros_like(a)
    z = torch.zeros(1, dtype=torch.float64, device=dev)
    cases = [
        (small.float(), None, a, b, c, d, z),                                   # solid not uint8
        (small, None, a, b, c.half(), d, z),                                    # X_out FP16
        (small, None, a, b, c, torch.zeros(10, device=dev), z),                 # X_ads_out too short
        (small, torch.zeros((3, 4, 4, 3), device=dev), a, b, c, d, z),          # u not 3 N
        (small, None, a, b, c, d, z.float()),                                   # Z_out not FP64
        (small, None, a.cpu(), b, c, d, z),                                     # X on the host
    ]
    for args in cases:
        sd, u, x, xa, xo, xao, zo = args
        with pytest.raises(mp.MPError) as e:
            mp.mp_step_noalloc(sd, u, 0.05, 0.0, 0.0, 0, x, xa, xo, xao, zo)
        assert e.value.code == mp.MP_EINVAL
