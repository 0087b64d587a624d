"""Thin Python binding of libmp (the C ABI in include/mp.h), with the same entry-point
names. It only marshals arguments: every step of the computation runs in the CUDA library.

Device buffers are passed as objects with a ``data_ptr()`` method (torch CUDA tensors) or
as integer addresses; host arrays are numpy arrays. Importing this module loads
``libmp.so`` and raises ImportError when it has not been built, so there is no silent
fallback to any other implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmp.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built: run paper_1303_2470_gb300.build.build() "
                      "(or __graft_entry__.build()) on a machine with the CUDA toolkit")
_lib = ctypes.CDLL(LIB_PATH)

MP_OK = 0
MP_EINVAL = -1
MP_ENOMEM = -2
MP_ECUDA = -3
MP_ENEGPROB = -4
MP_ENOTCONVERGED = -5
MP_ETIMEOUT = -6
MP_HOST = 0
MP_DEVICE = 1
MP_FP32 = 0
MP_FP64 = 1
MP_FP16 = 2
MP_ROUND_STOCHASTIC = 0
MP_ROUND_NEAREST = 1
MP_INIT_EQUILIBRIUM = 0
MP_INIT_UNIFORM = 1
MP_MAX_SPECIES = 32
MP_SCHEME_FLUX = 0
MP_SCHEME_DIRECT = 1
MP_VARIANT_RECOMPUTE = 1
MP_VARIANT_PERSISTENT = 2
MP_VARIANT_BLOCK128 = 4
MP_VARIANT_BLOCK512 = 8
MP_VARIANT_TILED = 16

_c_int, _c_i64, _c_dbl, _c_vp = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p


class mp_geometry(ctypes.Structure):
    _fields_ = [("nx", _c_int), ("ny", _c_int), ("nz", _c_int), ("solid", _c_vp), ("location", _c_int)]


class mp_options(ctypes.Structure):
    _fields_ = [("precision", _c_int), ("directions", _c_int), ("init_density", _c_int),
                ("allow_negative", _c_int), ("capacity", _c_i64), ("stream", _c_vp), ("rounding", _c_int),
                ("scheme", _c_int), ("autotune", _c_int), ("variant", _c_int)]


class mp_info_t(ctypes.Structure):
    _fields_ = [("n_nodes", _c_i64), ("n_fluid", _c_i64), ("n_interface", _c_i64),
                ("n_negative_links", _c_i64), ("t", _c_i64), ("n_species", _c_int),
                ("n_fields", _c_int), ("precision", _c_int)]


_dp = ctypes.POINTER(_c_dbl)
_lib.mp_default_options.argtypes = [ctypes.POINTER(mp_options)]
_lib.mp_default_options.restype = None
_lib.mp_last_error.restype = ctypes.c_char_p
_lib.mp_init.argtypes = [ctypes.POINTER(_c_vp), ctypes.POINTER(mp_geometry), _c_vp, _c_dbl, _c_dbl,
                         _c_dbl, ctypes.POINTER(mp_options)]
_lib.mp_init_batch.argtypes = [ctypes.POINTER(_c_vp), ctypes.POINTER(mp_geometry), _c_vp, _c_int,
                               _dp, _dp, _dp, ctypes.POINTER(mp_options)]
_lib.mp_step.argtypes = [_c_vp, _c_i64]
_lib.mp_vacf.argtypes = [_c_vp, _c_int, _c_int, _dp, _dp, _c_i64, ctypes.POINTER(_c_i64)]
_lib.mp_mass.argtypes = [_c_vp, _c_int, _dp]
_lib.mp_info.argtypes = [_c_vp, ctypes.POINTER(mp_info_t)]
_lib.mp_get_field.argtypes = [_c_vp, _c_int, _c_int, _dp, _dp]
_lib.mp_set_field.argtypes = [_c_vp, _c_int, _c_int, _dp, _dp]
_lib.mp_free.argtypes = [_c_vp]
_lib.mp_free.restype = None
_lib.lb_steady.argtypes = [ctypes.POINTER(mp_geometry), _dp, _c_dbl, _c_dbl, _c_i64, _c_i64, _c_vp, _c_vp,
                           _c_vp, _c_vp, ctypes.POINTER(_c_i64), _dp, _c_vp]
_lib.mp_classify.argtypes = [ctypes.POINTER(mp_geometry), _c_vp, ctypes.POINTER(_c_i64),
                             ctypes.POINTER(_c_i64), ctypes.POINTER(_c_i64), _c_vp]
_lib.mp_step_noalloc.argtypes = [_c_int, _c_int, _c_int, _c_vp, _c_vp, _c_dbl, _c_dbl, _c_dbl, _c_int,
                                 _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp]
_lib.mp_group_create.argtypes = [ctypes.POINTER(_c_vp), ctypes.POINTER(_c_vp), _c_int, _c_int, _c_int]
_lib.mp_group_create_ex.argtypes = [ctypes.POINTER(_c_vp), ctypes.POINTER(_c_vp), _c_int, _c_int, _c_int, _c_int]
_lib.mp_group_step.argtypes = [_c_vp, _c_i64]
_lib.mp_group_block_size.argtypes = [_c_vp]
_lib.mp_group_free.argtypes = [_c_vp]
_lib.mp_group_free.restype = None
_lib.mp_variant.argtypes = [_c_vp]
_lib.mp_variant.restype = ctypes.c_char_p
_lib.mp_group_variant.argtypes = [_c_vp]
_lib.mp_group_variant.restype = ctypes.c_char_p
_lib.mp_grid_wait_selftest.argtypes = [_c_int, _c_int, _c_int, _c_i64, _c_vp]
_f32, _c_i, _vp = ctypes.c_float, _c_int, _c_vp
_lib.sg_conv3d.argtypes = [_vp, _vp, _vp, _vp, _vp] + [_c_i] * 8 + [_vp]
_lib.sg_conv3d_wgrad.argtypes = [_vp, _vp, _vp, _vp] + [_c_i] * 6 + [_vp]
_lib.sg_check.argtypes = [_vp]
for _f in ("sg_pool2", "sg_pool2_grad", "sg_up2", "sg_up2_grad"):
    getattr(_lib, _f).argtypes = [_vp, _vp] + [_c_i] * 5 + [_vp]
_lib.sg_add.argtypes = [_vp, _vp, _vp, _c_i64, _vp]
_lib.sg_relu_grad.argtypes = [_vp, _vp, _c_i64, _vp]
_lib.sg_pack_input.argtypes = [_vp, _vp, _c_i, _c_i, _c_i, _c_i, _vp]
_lib.sg_unpack_output.argtypes = [_vp, _c_i, _vp, _vp, _vp, _c_i, _c_i, _c_i, _c_i, _f32, _f32, _vp]
_lib.sg_pack_target.argtypes = [_vp, _vp, _vp, _c_i, _c_i, _c_i, _c_i, _f32, _f32, _vp]
_lib.sg_mse.argtypes = [_vp, _c_i, _vp, _c_i, _vp, _vp, _vp, _c_i, _c_i, _c_dbl, _vp]
_lib.sg_adam.argtypes = [_vp, _vp, _vp, _vp, _c_i64, _f32, _f32, _f32, _f32, _c_i, _vp, _vp, _c_i, _c_i, _vp]
for _f in ("mp_init", "mp_init_batch", "mp_step", "mp_vacf", "mp_mass", "mp_info", "mp_get_field",
           "mp_set_field", "lb_steady", "mp_classify", "mp_step_noalloc", "mp_group_create", "mp_group_create_ex",
           "mp_grid_wait_selftest",
           "mp_group_step", "mp_group_block_size", "sg_conv3d", "sg_conv3d_wgrad", "sg_check", "sg_pool2",
           "sg_pool2_grad", "sg_up2", "sg_up2_grad", "sg_add", "sg_relu_grad", "sg_pack_input",
           "sg_unpack_output", "sg_pack_target", "sg_mse", "sg_adam"):
    getattr(_lib, _f).restype = _c_int


class MPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libmp status {code}: {msg}")
        self.code = code


class MPBufferError(MPError, ValueError):
    """A buffer that does not match the C ABI's documented layout, refused by the binding
    before any library call (status MP_EINVAL; also a ValueError)."""

    def __init__(self, msg):
        super().__init__(MP_EINVAL, msg)


def mp_last_error() -> str:
    return _lib.mp_last_error().decode()


def _check(rc):
    if rc != MP_OK:
        raise MPError(rc, mp_last_error())
    return rc


def _addr(buf):
    """Device address of a torch tensor / object with data_ptr(), or an int; None -> NULL."""
    if buf is None:
        return None
    if hasattr(buf, "data_ptr"):
        return int(buf.data_ptr())
    return int(buf)


def _check_dev_f32(buf, n, name):
    """A device FP32 buffer that must hold n values (None allowed). Torch tensors are
    checked (CUDA, float32, contiguous, at least n values), so that a wrong buffer raises
    here instead of being read or written out of bounds by the kernels; an integer address
    is the caller's responsibility."""
    if buf is not None and hasattr(buf, "numel") and hasattr(buf, "dtype"):
        if (not getattr(buf, "is_cuda", False) or str(buf.dtype) != "torch.float32" or not buf.is_contiguous()
                or buf.numel() < n):
            raise MPBufferError(f"{name}: needs a contiguous CUDA float32 tensor of at least {n} values, got "
                             f"shape {tuple(buf.shape)}, {buf.dtype}, on {getattr(buf, 'device', '?')}")


def _host_f64(a, n, name):
    """A host numpy float64 array of exactly n values that the library may read or write
    in place (C-contiguous)."""
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous and a.size == n):
        raise MPBufferError(f"{name}: needs a C-contiguous float64 numpy array of {n} values")
    return a.ctypes.data_as(_dp)


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


def make_geometry(solid):
    """mp_geometry for a solid mask: a numpy (host) or CUDA tensor (device) uint8 array
    shaped (nz, ny, nx). Returns (struct, keep-alive object)."""
    if hasattr(solid, "data_ptr") and getattr(solid, "is_cuda", False):
        if len(solid.shape) != 3 or str(solid.dtype) not in ("torch.uint8", "torch.bool"):
            raise ValueError(f"solid: needs a (nz, ny, nx) uint8 or bool tensor, got shape {tuple(solid.shape)}, "
                             f"{solid.dtype}")
        nz, ny, nx = solid.shape
        t = solid.contiguous()
        return mp_geometry(nx, ny, nz, t.data_ptr(), MP_DEVICE), t
    a = np.ascontiguousarray(solid, dtype=np.uint8)
    nz, ny, nx = a.shape
    return mp_geometry(nx, ny, nz, a.ctypes.data, MP_HOST), a


def mp_default_options() -> mp_options:
    o = mp_options()
    _lib.mp_default_options(ctypes.byref(o))
    return o


def _options(precision="fp32", directions="x", init_density="equilibrium", allow_negative=False,
             capacity=0, stream=None, rounding="stochastic", scheme="flux", autotune=False, variant=0):
    o = mp_default_options()
    o.scheme = {"flux": MP_SCHEME_FLUX, "direct": MP_SCHEME_DIRECT}[scheme]
    o.autotune = int(bool(autotune))
    o.variant = int(variant)
    o.precision = {"fp32": MP_FP32, "fp64": MP_FP64, "fp16": MP_FP16}[precision]
    o.rounding = {"stochastic": MP_ROUND_STOCHASTIC, "nearest": MP_ROUND_NEAREST}[rounding]
    o.directions = sum({"x": 1, "y": 2, "z": 4}[d] for d in directions)
    o.init_density = {"equilibrium": MP_INIT_EQUILIBRIUM, "uniform": MP_INIT_UNIFORM}[init_density]
    o.allow_negative = int(bool(allow_negative))
    o.capacity = int(capacity)
    o.stream = _stream(stream)
    return o


class Context:
    """Owning handle of an mp_ctx*; mp_free() runs on close() or garbage collection."""

    def __init__(self, ptr, shape, directions):
        self.ptr = ptr
        self.shape = shape
        self.directions = directions

    def close(self):
        if self.ptr:
            _lib.mp_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mp_init(solid, u, D_b, k_a, k_d, **options) -> Context:
    """mp_init of include/mp.h. solid: host numpy or device tensor (nz,ny,nx) uint8;
    u: device FP32 buffer of 3*N values (SoA) or None. Options: precision ("fp32"/"fp64"/"fp16"),
    scheme ("flux"/"direct"), autotune (direct scheme), variant (MP_VARIANT_* flags),
    rounding of fp16 storage ("stochastic"/"nearest"),
    directions (e.g. "x", "xz"), init_density ("equilibrium"/"uniform"), allow_negative,
    capacity, stream."""
    return mp_init_batch(solid, u, [D_b], [k_a], [k_d], **options)


def mp_init_batch(solid, u, D_b, k_a, k_d, **options) -> Context:
    g, keep = make_geometry(solid)
    Db = np.ascontiguousarray(D_b, dtype=np.float64)
    ka = np.ascontiguousarray(k_a, dtype=np.float64)
    kd = np.ascontiguousarray(k_d, dtype=np.float64)
    if not (Db.shape == ka.shape == kd.shape and Db.ndim == 1):
        raise ValueError("D_b, k_a, k_d must be 1-D arrays of equal length")
    o = _options(**options)
    _check_dev_f32(u, 3 * g.nx * g.ny * g.nz, "u")
    out = _c_vp()
    _check(_lib.mp_init_batch(ctypes.byref(out), ctypes.byref(g), _addr(u), len(Db),
                              Db.ctypes.data_as(_dp), ka.ctypes.data_as(_dp), kd.ctypes.data_as(_dp),
                              ctypes.byref(o)))
    del keep
    return Context(out, (g.nz, g.ny, g.nx), options.get("directions", "x"))


def mp_step(ctx: Context, n: int):
    _check(_lib.mp_step(ctx.ptr, int(n)))


def mp_variant(ctx: Context) -> str:
    """How mp_step runs this context ("flux", or the direct scheme's launch form, link terms
    and block size)."""
    return _lib.mp_variant(ctx.ptr).decode()


def mp_grid_wait_selftest(n_blocks: int, rounds: int, unreachable: bool, timeout_ns: int, stream=None):
    """mp_grid_wait_selftest of include/mp.h; raises MPError (code MP_ETIMEOUT) when a wait
    gave up."""
    _check(_lib.mp_grid_wait_selftest(int(n_blocks), int(rounds), int(bool(unreachable)), int(timeout_ns),
                                      _stream(stream)))


def mp_vacf(ctx: Context, species: int = 0, direction: int = 0, cap: int | None = None):
    """Returns (Z, D), numpy float64 arrays of the available time points (t = 0..T)."""
    n = _c_i64()
    _check(_lib.mp_vacf(ctx.ptr, species, direction, None, None, 0, ctypes.byref(n)))
    T = n.value if cap is None else min(n.value, cap)
    Z = np.zeros(T)
    D = np.zeros(T)
    _check(_lib.mp_vacf(ctx.ptr, species, direction, Z.ctypes.data_as(_dp), D.ctypes.data_as(_dp), T,
                        ctypes.byref(n)))
    return Z, D


def mp_vacf_into(ctx: Context, species: int, direction: int, Z: np.ndarray, D: np.ndarray) -> int:
    """mp_vacf into caller-owned host arrays (e.g. pinned); returns the time points available."""
    n = _c_i64()
    m = min(Z.size, D.size)
    _check(_lib.mp_vacf(ctx.ptr, species, direction, _host_f64(Z[:m], m, "Z"), _host_f64(D[:m], m, "D"), m,
                        ctypes.byref(n)))
    return n.value


def mp_mass(ctx: Context, species: int = 0) -> np.ndarray:
    out = np.zeros(3)
    _check(_lib.mp_mass(ctx.ptr, species, out.ctypes.data_as(_dp)))
    return out


def mp_info(ctx: Context) -> dict:
    i = mp_info_t()
    _check(_lib.mp_info(ctx.ptr, ctypes.byref(i)))
    return {k: getattr(i, k) for k, _ in mp_info_t._fields_}


def mp_get_field(ctx: Context, species: int = 0, field: int = 0):
    """(free, adsorbed) dense float64 arrays shaped (nz, ny, nx)."""
    fr = np.zeros(ctx.shape)
    ad = np.zeros(ctx.shape)
    _check(_lib.mp_get_field(ctx.ptr, species, field, fr.ctypes.data_as(_dp), ad.ctypes.data_as(_dp)))
    return fr, ad


def mp_set_field(ctx: Context, species: int, field: int, free, ads=None):
    n = int(np.prod(ctx.shape))
    fr = np.ascontiguousarray(free, dtype=np.float64)
    ad = None if ads is None else np.ascontiguousarray(ads, dtype=np.float64)
    _check(_lib.mp_set_field(ctx.ptr, species, field, _host_f64(fr, n, "free"),
                             _host_f64(ad, n, "ads") if ad is not None else None))


def mp_classify(solid, stream=None):
    """Node classes (0 solid, 1 fluid, 2 interfacial, +4 in the largest fluid cluster) as a
    uint8 array shaped like `solid`, and the counts (n_fluid, n_interface, n_cluster)."""
    g, keep = make_geometry(solid)
    cls = np.zeros((g.nz, g.ny, g.nx), dtype=np.uint8)
    nf, ni, nc = _c_i64(), _c_i64(), _c_i64()
    _check(_lib.mp_classify(ctypes.byref(g), cls.ctypes.data, ctypes.byref(nf), ctypes.byref(ni),
                            ctypes.byref(nc), _stream(stream)))
    del keep
    return cls, (nf.value, ni.value, nc.value)


def _device_of(buf):
    return str(getattr(buf, "device", "?"))


def mp_step_noalloc(solid, u, D_b, k_a, k_d, direction, X, X_ads, X_out, X_ads_out, Z_out,
                    stream=None):
    """mp_step_noalloc of include/mp.h: one step of one field on caller-owned device arrays
    (torch CUDA tensors), allocating nothing. solid: uint8 (nz, ny, nx); u: FP32 (3, nz, ny,
    nx) or None; X, X_ads, X_out, X_ads_out: FP32 (nz, ny, nx); Z_out: one FP64 element.
    Every tensor is checked against that layout (CUDA, dtype, contiguity, size, one device)
    before the call, which then runs with that device current."""
    if not (hasattr(solid, "data_ptr") and getattr(solid, "is_cuda", False) and len(solid.shape) == 3
            and str(solid.dtype) in ("torch.uint8", "torch.bool") and solid.is_contiguous()):
        raise MPBufferError(f"solid: needs a contiguous CUDA uint8 tensor (nz, ny, nx), got "
                            f"{getattr(solid, 'shape', '?')}, {getattr(solid, 'dtype', '?')}")
    nz, ny, nx = solid.shape
    N = nx * ny * nz
    bufs = [("solid", solid)]
    for name, buf, n in (("u", u, 3 * N), ("X", X, N), ("X_ads", X_ads, N), ("X_out", X_out, N),
                         ("X_ads_out", X_ads_out, N)):
        if buf is None and name != "u":
            raise MPBufferError(f"{name}: a CUDA float32 tensor of {n} values is required")
        if buf is not None and not hasattr(buf, "numel"):
            raise MPBufferError(f"{name}: needs a CUDA tensor")
        _check_dev_f32(buf, n, name)
        if buf is not None:
            bufs.append((name, buf))
    if not (hasattr(Z_out, "numel") and getattr(Z_out, "is_cuda", False) and str(Z_out.dtype) == "torch.float64"
            and Z_out.numel() >= 1):
        raise MPBufferError("Z_out: needs a CUDA float64 tensor of at least one element")
    bufs.append(("Z_out", Z_out))
    devs = {_device_of(b) for _, b in bufs}
    if len(devs) != 1:
        raise MPBufferError(f"all buffers must be on one device, got {sorted(devs)}")
    import torch
    with torch.cuda.device(solid.device):
        _check(_lib.mp_step_noalloc(nx, ny, nz, _addr(solid), _addr(u), float(D_b), float(k_a), float(k_d),
                                    int(direction), _addr(X), _addr(X_ads), _addr(X_out), _addr(X_ads_out),
                                    _addr(Z_out), _stream(stream)))


class Group:
    """Owning handle of an mp_group*; keeps its contexts alive and frees first."""

    def __init__(self, ptr, ctxs):
        self.ptr = ptr
        self.ctxs = list(ctxs)

    def close(self):
        if self.ptr:
            _lib.mp_group_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mp_group_create(ctxs, graph_steps: int = 0, autotune: bool = False, variant: int = 0) -> Group:
    """mp_group_create_ex of include/mp.h over a list of Context objects (variant: MP_VARIANT_*
    flags of a direct group without autotune)."""
    arr = (_c_vp * len(ctxs))(*[c.ptr for c in ctxs])
    out = _c_vp()
    _check(_lib.mp_group_create_ex(ctypes.byref(out), arr, len(ctxs), int(graph_steps), int(bool(autotune)),
                                   int(variant)))
    return Group(out, ctxs)


def mp_group_step(group: Group, n: int):
    _check(_lib.mp_group_step(group.ptr, int(n)))


def mp_group_block_size(group: Group) -> int:
    return int(_lib.mp_group_block_size(group.ptr))


def mp_group_variant(group: Group) -> str:
    return _lib.mp_group_variant(group.ptr).decode()


def mp_group_free(group: Group):
    group.close()


def mp_free(ctx: Context):
    ctx.close()


def lb_steady(solid, force, u_out, tau=1.0, tol=1e-7, max_steps=1_000_000, check_every=100,
              u_init=None, stream=None, raise_on_unconverged=False, rho_init=None, rho_out=None):
    """lb_steady of include/mp.h; u_out (and u_init) are device FP32 buffers of 3*N values,
    rho_init and rho_out of N values. Returns (steps, residual, converged)."""
    g, keep = make_geometry(solid)
    F = np.ascontiguousarray(force, dtype=np.float64)
    if F.shape != (3,):
        raise ValueError("force: needs three components")
    N = g.nx * g.ny * g.nz
    if u_out is None:
        raise ValueError("u_out: a device FP32 buffer of 3*N values is required")
    bufs = ((u_init, 3 * N, "u_init"), (rho_init, N, "rho_init"), (u_out, 3 * N, "u_out"), (rho_out, N, "rho_out"))
    for buf, n, name in bufs:
        _check_dev_f32(buf, n, name)
    steps = _c_i64()
    res = _c_dbl()
    rc = _lib.lb_steady(ctypes.byref(g), F.ctypes.data_as(_dp), float(tau), float(tol), int(max_steps),
                        int(check_every), *(_addr(b[0]) for b in bufs), ctypes.byref(steps), ctypes.byref(res),
                        _stream(stream))
    del keep
    if rc == MP_ENOTCONVERGED and not raise_on_unconverged:
        return steps.value, res.value, False
    _check(rc)
    return steps.value, res.value, True


# ---- kernels of the learned LB warm start (include/surrogate.h) ------------------------
def sg_conv3d(x, w, bias, y, yf, B, D, H, W, K, N, sign=1, relu=False, stream=None):
    _check(_lib.sg_conv3d(_addr(x), _addr(w), _addr(bias), _addr(y), _addr(yf), B, D, H, W, K, N, sign,
                          int(bool(relu)), _stream(stream)))


def sg_check(stream=None):
    """sg_check of include/surrogate.h: raises MPError (MP_ETIMEOUT) if a tensor-core
    convolution since the last check gave up a bounded wait."""
    _check(_lib.sg_check(_stream(stream)))


def sg_conv3d_wgrad(x, dy, dw, dbias, B, D, H, W, Cin, Cout, stream=None):
    _check(_lib.sg_conv3d_wgrad(_addr(x), _addr(dy), _addr(dw), _addr(dbias), B, D, H, W, Cin, Cout,
                                _stream(stream)))


def sg_pool2(x, y, B, D, H, W, C, stream=None):
    _check(_lib.sg_pool2(_addr(x), _addr(y), B, D, H, W, C, _stream(stream)))


def sg_pool2_grad(dy, dx, B, D, H, W, C, stream=None):
    _check(_lib.sg_pool2_grad(_addr(dy), _addr(dx), B, D, H, W, C, _stream(stream)))


def sg_up2(x, y, B, D, H, W, C, stream=None):
    _check(_lib.sg_up2(_addr(x), _addr(y), B, D, H, W, C, _stream(stream)))


def sg_up2_grad(dy, dx, B, D, H, W, C, stream=None):
    _check(_lib.sg_up2_grad(_addr(dy), _addr(dx), B, D, H, W, C, _stream(stream)))


def sg_add(a, b, y, n, stream=None):
    _check(_lib.sg_add(_addr(a), _addr(b), _addr(y), int(n), _stream(stream)))


def sg_relu_grad(act, g, n, stream=None):
    _check(_lib.sg_relu_grad(_addr(act), _addr(g), int(n), _stream(stream)))


def sg_pack_input(cls, x, nx, ny, nz, axis, stream=None):
    _check(_lib.sg_pack_input(_addr(cls), _addr(x), nx, ny, nz, axis, _stream(stream)))


def sg_unpack_output(y, ldy, cls, u, rho, nx, ny, nz, axis, scale_u, scale_rho=0.0, stream=None):
    _check(_lib.sg_unpack_output(_addr(y), ldy, _addr(cls), _addr(u), _addr(rho), nx, ny, nz, axis,
                                 float(scale_u), float(scale_rho), _stream(stream)))


def sg_pack_target(u, rho, t, nx, ny, nz, axis, scale_u, scale_rho, stream=None):
    _check(_lib.sg_pack_target(_addr(u), _addr(rho), _addr(t), nx, ny, nz, axis, float(scale_u),
                               float(scale_rho), _stream(stream)))


def sg_mse(y, ldy, t, nc, x, dy, loss, B, V, n_fluid, stream=None):
    _check(_lib.sg_mse(_addr(y), ldy, _addr(t), nc, _addr(x), _addr(dy), _addr(loss), B, V, float(n_fluid),
                       _stream(stream)))


def sg_adam(p, g, m, v, n, lr, b1, b2, eps, t, wf=None, wb=None, cin=0, cout=0, stream=None):
    _check(_lib.sg_adam(_addr(p), _addr(g), _addr(m), _addr(v), int(n), float(lr), float(b1), float(b2),
                        float(eps), int(t), _addr(wf), _addr(wb), cin, cout, _stream(stream)))

