"""FP64 CPU oracle of the sorption-modified moment-propagation method (arXiv:1303.2470).

TEST INFRASTRUCTURE ONLY. This package is the plain, slow, obviously correct statement of
what the GPU library computes. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import it; the product package never
does, and the two share no code, constants or helpers. The arithmetic lives in
``mp_oracle.c`` (plain C, FP64, one node at a time); this module compiles it with gcc and
marshals numpy arrays through ctypes.

Sections cited are those of the paper: Sec. "Algorithm" defines the propagation
(Eq. propagated_quantity), the link probability p_i, D_b = lambda c_s^2 dt / 4, the
sorption update (Eqs. Pads and newP), the Boltzmann weights and the VACF sum; the
Introduction defines D(t) and K from the VACF (Eqs. D_t_from_vacf, K_from_vacf).
Readings R1-R6 of the paper are listed at the top of ``mp_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile mp_oracle.c into liboracle.so (in place). FP contraction is off so that x86
    and Arm hosts round identically."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.or_link_prob.restype = ctypes.c_double
        lib.or_mean_step.restype = ctypes.c_double
        lib.or_vacf_z0.restype = ctypes.c_double
        lib.or_vacf.restype = ctypes.c_double
        lib.or_sum.restype = ctypes.c_double
        _lib = lib
    return _lib


class _OrMp(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("solid", _u8p), ("u", _dp), ("D_b", ctypes.c_double),
                ("k_a", ctypes.c_double), ("k_d", ctypes.c_double)]


def _ptr(a, t):
    return a.ctypes.data_as(t)


def d3q19():
    """The oracle's own D3Q19 table: (c[19,3], w[19], opp[19])."""
    lib = _load()
    c = np.zeros((19, 3), dtype=np.int32)
    w = np.zeros(19)
    opp = np.zeros(19, dtype=np.int32)
    lib.or_d3q19(c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _ptr(w, _dp),
                 opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return c, w, opp


def classify(solid: np.ndarray):
    """Node classes (0 solid, 1 fluid off the interface, 2 interfacial) of a solid mask
    shaped (nz, ny, nx); returns (cls, n_fluid, n_iface)."""
    lib = _load()
    s = np.ascontiguousarray(solid, dtype=np.uint8)
    nz, ny, nx = s.shape
    cls = np.zeros_like(s)
    nf = ctypes.c_int64()
    ni = ctypes.c_int64()
    lib.or_classify(nx, ny, nz, _ptr(s, _u8p), _ptr(cls, _u8p), ctypes.byref(nf), ctypes.byref(ni))
    return cls, nf.value, ni.value


@dataclass
class Problem:
    """One tracer species in one medium. solid: (nz, ny, nx) uint8; u: (3, nz, ny, nx)
    float64 or None (fluid at rest); D_b, k_a, k_d in lattice units."""
    solid: np.ndarray
    u: np.ndarray | None
    D_b: float
    k_a: float
    k_d: float

    def __post_init__(self):
        self.solid = np.ascontiguousarray(self.solid, dtype=np.uint8)
        if self.u is not None:
            self.u = np.ascontiguousarray(self.u, dtype=np.float64)
            assert self.u.shape == (3,) + self.solid.shape

    @property
    def shape(self):
        return self.solid.shape

    @property
    def N(self):
        return int(self.solid.size)

    def _c(self):
        nz, ny, nx = self.solid.shape
        s = _OrMp()
        s.nx, s.ny, s.nz = nx, ny, nz
        s.solid = _ptr(self.solid, _u8p)
        s.u = _ptr(self.u, _dp) if self.u is not None else _dp()
        s.D_b, s.k_a, s.k_d = float(self.D_b), float(self.k_a), float(self.k_d)
        return s


def link_prob(p: Problem, n: int, i: int) -> float:
    """p_i at linear node n (oracle link order, see d3q19())."""
    return _load().or_link_prob(ctypes.byref(p._c()), ctypes.c_int64(n), i)


def mean_step(p: Problem, n: int, g: int) -> float:
    """sum_i p_i(r) c_ig at linear node n."""
    return _load().or_mean_step(ctypes.byref(p._c()), ctypes.c_int64(n), g)


def propagate(p: Problem, X: np.ndarray, Xa: np.ndarray):
    """One MP + sorption step of one field (Eqs. propagated_quantity, Pads, newP with
    reading R1). X, Xa dense (nz, ny, nx) float64; returns (X', Xa')."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    Xa = np.ascontiguousarray(Xa, dtype=np.float64)
    Xn = np.zeros_like(X)
    Xan = np.zeros_like(X)
    _load().or_mp_propagate(ctypes.byref(p._c()), _ptr(X, _dp), _ptr(Xa, _dp), _ptr(Xn, _dp),
                            _ptr(Xan, _dp))
    return Xn, Xan


def equilibrium(p: Problem):
    """Boltzmann weights (free pi, adsorbed pi_ads), normalised to total mass one."""
    pi = np.zeros(p.shape)
    pa = np.zeros(p.shape)
    rc = _load().or_equilibrium(ctypes.byref(p._c()), _ptr(pi, _dp), _ptr(pa, _dp))
    if rc != 0:
        raise ValueError("no equilibrium: k_a > 0 with k_d = 0")
    return pi, pa


def moment_init(p: Problem, g: int, pi: np.ndarray) -> np.ndarray:
    pi = np.ascontiguousarray(pi, dtype=np.float64)
    out = np.zeros(p.shape)
    _load().or_moment_init(ctypes.byref(p._c()), g, _ptr(pi, _dp), _ptr(out, _dp))
    return out


def vacf_z0(p: Problem, g: int, pi: np.ndarray) -> float:
    pi = np.ascontiguousarray(pi, dtype=np.float64)
    return _load().or_vacf_z0(ctypes.byref(p._c()), g, _ptr(pi, _dp))


def vacf(p: Problem, g: int, Pg: np.ndarray) -> float:
    Pg = np.ascontiguousarray(Pg, dtype=np.float64)
    return _load().or_vacf(ctypes.byref(p._c()), g, _ptr(Pg, _dp))


@dataclass
class Run:
    Z: np.ndarray
    D: np.ndarray
    mass_free: np.ndarray
    mass_ads: np.ndarray
    iface_free: np.ndarray
    P: np.ndarray
    Pa: np.ndarray
    Pg: np.ndarray
    Pga: np.ndarray


def run(p: Problem, g: int = 0, nsteps: int = 0, init: str = "equilibrium") -> Run:
    """Initialise and advance nsteps steps; series have nsteps+2 entries (t = 0..nsteps+1).
    init = "equilibrium" (density starts at the Boltzmann weights) or "uniform" (density
    starts uniform over the free fluid with no adsorbed tracer)."""
    mode = {"equilibrium": 0, "uniform": 1}[init]
    T = nsteps + 2
    Z, D, mf, ma, mi = (np.zeros(T) for _ in range(5))
    P, Pa, Pg, Pga = (np.zeros(p.shape) for _ in range(4))
    rc = _load().or_mp_run(ctypes.byref(p._c()), g, mode, ctypes.c_int64(nsteps), _ptr(Z, _dp),
                           _ptr(D, _dp), _ptr(mf, _dp), _ptr(ma, _dp), _ptr(mi, _dp),
                           _ptr(P, _dp), _ptr(Pa, _dp), _ptr(Pg, _dp), _ptr(Pga, _dp))
    if rc != 0:
        raise ValueError("oracle run rejected its input")
    return Run(Z, D, mf, ma, mi, P, Pa, Pg, Pga)


def lb_init(solid: np.ndarray, u0: np.ndarray | None = None, rho0: np.ndarray | None = None) -> np.ndarray:
    """Populations f[19, nz, ny, nx] = f^eq(rho0, u0) (rho0 = 1 and u0 = 0 by default;
    oracle link order)."""
    s = np.ascontiguousarray(solid, dtype=np.uint8)
    nz, ny, nx = s.shape
    f = np.zeros((19,) + s.shape)
    u0c = None if u0 is None else np.ascontiguousarray(u0, dtype=np.float64)
    r0c = None if rho0 is None else np.ascontiguousarray(rho0, dtype=np.float64)
    _load().or_lb_init(nx, ny, nz, _ptr(s, _u8p), _ptr(u0c, _dp) if u0c is not None else _dp(),
                       _ptr(r0c, _dp) if r0c is not None else _dp(), _ptr(f, _dp))
    return f


def largest_cluster(solid):
    """(in_cluster uint8[...], size): the largest D3Q19-connected cluster of fluid nodes."""
    s = np.ascontiguousarray(solid, dtype=np.uint8)
    nz, ny, nx = s.shape
    out = np.zeros_like(s)
    size = ctypes.c_int64()
    if _load().or_largest_cluster(nx, ny, nz, _ptr(s, _u8p), _ptr(out, _u8p), ctypes.byref(size)) != 0:
        raise MemoryError("oracle cluster search")
    return out, size.value


def lb_step(solid, f, force, tau=1.0, forced=None):
    """One BGK + Guo + halfway bounce-back step; returns (f', u[3,nz,ny,nx]). The force
    acts where `forced` is nonzero (on every fluid node when None)."""
    s = np.ascontiguousarray(solid, dtype=np.uint8)
    nz, ny, nx = s.shape
    f = np.ascontiguousarray(f, dtype=np.float64)
    fo = np.zeros_like(f)
    u = np.zeros((3,) + s.shape)
    F = (ctypes.c_double * 3)(*[float(v) for v in force])
    fm = None if forced is None else np.ascontiguousarray(forced, dtype=np.uint8)
    _load().or_lb_step(nx, ny, nz, _ptr(s, _u8p), _ptr(fm, _u8p) if fm is not None else _u8p(), F,
                       ctypes.c_double(tau), _ptr(f, _dp), _ptr(fo, _dp), _ptr(u, _dp))
    return fo, u


def lb_steady(solid, force, tau=1.0, tol=1e-7, max_steps=200000, check_every=100, u_init=None,
              rho_init=None, with_rho=False, with_f=False):
    """Steady BGK flow, force on the largest fluid cluster, started from f^eq(rho_init, u_init)
    (rest and unit density by default); returns (u[3,nz,ny,nx], steps, residual, converged),
    plus the final density rho[nz,ny,nx] (0 on solids) when with_rho, plus the final
    populations f[19,nz,ny,nx] when with_f."""
    s = np.ascontiguousarray(solid, dtype=np.uint8)
    nz, ny, nx = s.shape
    u = np.zeros((3,) + s.shape)
    rho = np.zeros(s.shape)
    F = (ctypes.c_double * 3)(*[float(v) for v in force])
    steps = ctypes.c_int64()
    res = ctypes.c_double()
    fo = np.zeros((19,) + s.shape) if with_f else None
    ui = None if u_init is None else np.ascontiguousarray(u_init, dtype=np.float64)
    ri = None if rho_init is None else np.ascontiguousarray(rho_init, dtype=np.float64)
    rc = _load().or_lb_steady(nx, ny, nz, _ptr(s, _u8p), F, ctypes.c_double(tau),
                              ctypes.c_double(tol), ctypes.c_int64(max_steps),
                              ctypes.c_int64(check_every),
                              _ptr(ui, _dp) if ui is not None else _dp(),
                              _ptr(ri, _dp) if ri is not None else _dp(), _ptr(u, _dp), _ptr(rho, _dp),
                              ctypes.byref(steps), ctypes.byref(res), _ptr(fo, _dp) if with_f else _dp())
    if rc < 0:
        raise ValueError("oracle LB rejected its input")
    out = (u, steps.value, res.value, rc == 0)
    if with_rho:
        out = out + (rho,)
    return out + (fo,) if with_f else out
