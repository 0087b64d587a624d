"""The Python binding refuses buffers that do not match the C ABI's documented layout
before any library call (CPU; nothing reaches the kernels): wrong device, dtype, size or
contiguity of device buffers, and host arrays the library would read or write in place."""
import numpy as np
import pytest
import torch


@pytest.fixture(scope="module")
def mp():
    from paper_1303_2470_gb300 import build as b
    b.build()
    from paper_1303_2470_gb300 import mp as m
    return m


class FakeCuda:
    """Stands in for a CUDA tensor on a machine without a GPU; its address is never used
    because every case below is rejected first."""

    def __init__(self, shape, dtype=torch.float32, contiguous=True):
        self.shape = tuple(shape)
        self.dtype = dtype
        self.device = "cuda:0"
        self.is_cuda = True
        self._contiguous = contiguous

    def numel(self):
        return int(np.prod(self.shape))

    def is_contiguous(self):
        return self._contiguous

    def data_ptr(self):
        raise AssertionError("address requested for a buffer that should have been rejected")


class FakeCtx:
    def __init__(self, shape):
        self.ptr = None
        self.shape = shape


def test_lb_steady_rejects_mismatched_buffers(mp):
    solid = np.zeros((4, 5, 6), np.uint8)
    N = solid.size
    F = (1e-5, 0.0, 0.0)
    for bad in (FakeCuda((3 * N - 1,)),                       # too small
                FakeCuda((3 * N,), dtype=torch.float64),      # wrong dtype
                FakeCuda((3 * N,), contiguous=False),         # not dense SoA
                torch.zeros(3 * N, dtype=torch.float32)):     # host memory
        with pytest.raises(ValueError, match="u_out"):
            mp.lb_steady(solid, F, bad)
    good = FakeCuda((3, 4, 5, 6))
    with pytest.raises(ValueError, match="rho_out"):
        mp.lb_steady(solid, F, good, rho_out=FakeCuda((N - 1,)))
    with pytest.raises(ValueError, match="u_init"):
        mp.lb_steady(solid, F, good, u_init=FakeCuda((N,)))
    with pytest.raises(ValueError, match="rho_init"):
        mp.lb_steady(solid, F, good, rho_init=FakeCuda((N,), dtype=torch.float16))
    with pytest.raises(ValueError, match="force"):
        mp.lb_steady(solid, (1e-5, 0.0), good)
    with pytest.raises(ValueError, match="u_out"):
        mp.lb_steady(solid, F, None)


def test_mp_init_and_geometry_reject_mismatched_buffers(mp):
    solid = np.zeros((4, 5, 6), np.uint8)
    with pytest.raises(ValueError, match="u"):
        mp.mp_init(solid, FakeCuda((3 * solid.size - 3,)), 0.05, 0.0, 0.0)
    with pytest.raises(ValueError, match="solid"):
        mp.make_geometry(FakeCuda((4, 5, 6), dtype=torch.int32))
    with pytest.raises(ValueError, match="solid"):
        mp.make_geometry(FakeCuda((20, 6), dtype=torch.uint8))


def test_host_arrays_written_or_read_in_place_are_checked(mp):
    ctx = FakeCtx((4, 5, 6))
    with pytest.raises(ValueError, match="Z"):
        mp.mp_vacf_into(ctx, 0, 0, np.zeros(10, np.float32), np.zeros(10))
    with pytest.raises(ValueError, match="D"):
        mp.mp_vacf_into(ctx, 0, 0, np.zeros(10), np.zeros(20)[::2])
    with pytest.raises(ValueError, match="free"):
        mp.mp_set_field(ctx, 0, 0, np.zeros((4, 5, 5)))
    with pytest.raises(ValueError, match="ads"):
        mp.mp_set_field(ctx, 0, 0, np.zeros((4, 5, 6)), np.zeros(7))


def test_documented_buffers_pass(mp):
    # the shapes every caller uses: u (3, nz, ny, nx), rho (nz, ny, nx), FP32, dense
    for shape, n in (((3, 4, 5, 6), 3 * 120), ((4, 5, 6), 120), ((3 * 120 + 8,), 3 * 120)):
        mp._check_dev_f32(FakeCuda(shape), n, "buf")
    mp._check_dev_f32(None, 10, "buf")
    assert mp._host_f64(np.zeros(7), 7, "Z") is not None


def test_noalloc_binding_refuses_mismatched_buffers(mp):
    solid = FakeCuda((4, 5, 6), dtype=torch.uint8)
    N = 4 * 5 * 6
    ok = [FakeCuda((4, 5, 6)) for _ in range(4)]
    z = FakeCuda((1,), dtype=torch.float64)
    other = FakeCuda((4, 5, 6))
    other.device = "cuda:1"
    cases = [
        ((FakeCuda((4, 5, 6), dtype=torch.int32), None, *ok, z), "solid"),
        ((FakeCuda((N,), dtype=torch.uint8), None, *ok, z), "solid"),
        ((solid, FakeCuda((3 * N - 1,)), *ok, z), "u"),
        ((solid, None, FakeCuda((4, 5, 6), dtype=torch.float16), *ok[1:], z), "X"),
        ((solid, None, *ok[:3], FakeCuda((N - 1,)), z), "X_ads_out"),
        ((solid, None, *ok[:2], FakeCuda((4, 5, 6), contiguous=False), ok[3], z), "X_out"),
        ((solid, None, *ok, FakeCuda((1,), dtype=torch.float32)), "Z_out"),
        ((solid, None, *ok[:3], other, z), "one device"),
        ((solid, None, ok[0], None, *ok[2:], z), "X_ads"),
    ]
    for (sd, u, x, xa, xo, xao, zo), what in cases:
        with pytest.raises(mp.MPError, match=what) as e:
            mp.mp_step_noalloc(sd, u, 0.05, 0.0, 0.0, 0, x, xa, xo, xao, zo)
        assert e.value.code == mp.MP_EINVAL and isinstance(e.value, ValueError)
