"""FP64 CPU oracle of the WENO-Wombat MHD hot path (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg (``bench.py`` cpu_baseline / ``--impl reference``)
may import this package.  The product path never does, and the oracle shares
no code with the CUDA library.

Arrays follow the library's layout: cell fields ``U[8, nz, ny, nx]`` (rho, mx,
my, mz, Bx, By, Bz, E) and face fields ``bx, by, bz [nz, ny, nx]`` (lower
faces), all float64, periodic.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)


class OrcGrid(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
        ("gamma", ctypes.c_double), ("emf_mode", ctypes.c_int), ("weights", ctypes.c_int),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        d, i = ctypes.c_double, ctypes.c_int
        G = ctypes.POINTER(OrcGrid)
        L.orc_phi_n.restype = d
        L.orc_phi_n.argtypes = [d, d, d, d]
        L.orc_phi_n_z.restype = d
        L.orc_phi_n_z.argtypes = [d, d, d, d]
        L.orc_weno_weights_z.argtypes = [d, d, d, d, _dp, _dp, _dp]
        L.orc_weno_weights.argtypes = [d, d, d, d, _dp, _dp, _dp]
        L.orc_cons_to_prim.argtypes = [_dp, d, _dp]
        L.orc_prim_to_cons.argtypes = [_dp, d, _dp]
        L.orc_flux_n.argtypes = [_dp, d, _dp]
        L.orc_wave_speeds.argtypes = [_dp, d, _dp, _dp, _dp]
        L.orc_eigen.restype = i
        L.orc_eigen.argtypes = [_dp, d, _dp, _dp, _dp]
        L.orc_interface_flux.argtypes = [_dp, d, _dp]
        L.orc_cell_b.argtypes = [G, _dp, _dp, _dp, _dp]
        L.orc_face_fluxes.argtypes = [G, _dp, i, _dp]
        L.orc_rhs.argtypes = [G, _dp, _dp, _dp, _dp, _dp, _dp]
        L.orc_ssprk3_step.argtypes = [G, d, _dp, _dp, _dp, _dp]
        L.orc_rk4_step.argtypes = [G, d, _dp, _dp, _dp, _dp]
        L.orc_cfl_speed.restype = d
        L.orc_cfl_speed.argtypes = [G, _dp]
        L.orc_cfl_dt.restype = d
        L.orc_cfl_dt.argtypes = [G, d, _dp]
        L.orc_totals.argtypes = [G, _dp, _dp]
        L.orc_div_b.argtypes = [G, _dp, _dp, _dp, _dp]
        L.orc_num_threads.restype = i
        L.orc_set_num_threads.argtypes = [i]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _vec(x, n):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(n))
    return a


# ---------------------------------------------------------------- point-wise
def phi_n(a, b, c, d) -> float:
    return lib().orc_phi_n(float(a), float(b), float(c), float(d))


def phi_n_z(a, b, c, d) -> float:
    return lib().orc_phi_n_z(float(a), float(b), float(c), float(d))


def weno_weights_z(a, b, c, d):
    w = [ctypes.c_double() for _ in range(3)]
    lib().orc_weno_weights_z(float(a), float(b), float(c), float(d), *[ctypes.byref(x) for x in w])
    return tuple(x.value for x in w)


def weno_weights(a, b, c, d):
    w = [ctypes.c_double() for _ in range(3)]
    lib().orc_weno_weights(float(a), float(b), float(c), float(d),
                           *[ctypes.byref(x) for x in w])
    return tuple(x.value for x in w)


def cons_to_prim(U, gamma=5.0 / 3.0):
    U = _vec(U, 8)
    W = np.empty(8)
    lib().orc_cons_to_prim(_p(U), gamma, _p(W))
    return W


def prim_to_cons(W, gamma=5.0 / 3.0):
    W = _vec(W, 8)
    U = np.empty(8)
    lib().orc_prim_to_cons(_p(W), gamma, _p(U))
    return U


def flux_n(U, gamma=5.0 / 3.0):
    U = _vec(U, 8)
    F = np.empty(8)
    lib().orc_flux_n(_p(U), gamma, _p(F))
    return F


def wave_speeds(W, gamma=5.0 / 3.0):
    W = _vec(W, 8)
    r = [ctypes.c_double() for _ in range(3)]
    lib().orc_wave_speeds(_p(W), gamma, *[ctypes.byref(x) for x in r])
    return tuple(x.value for x in r)


def eigen(W, gamma=5.0 / 3.0):
    """(lambda[7], RU[7,7], LU[7,7], status) at primitive state W (normal frame)."""
    W = _vec(W, 8)
    lam = np.empty(7)
    RU = np.empty(49)
    LU = np.empty(49)
    st = lib().orc_eigen(_p(W), gamma, _p(lam), _p(RU), _p(LU))
    return lam, RU.reshape(7, 7), LU.reshape(7, 7), st


def interface_flux(Us, gamma=5.0 / 3.0):
    """Eq. FWENO flux at i+1/2 from the stencil cells i-2..i+3 (6x8, normal frame)."""
    Us = _vec(Us, 48)
    F = np.empty(8)
    lib().orc_interface_flux(_p(Us), gamma, _p(F))
    return F


# ---------------------------------------------------------------- grid level
@dataclass
class Grid:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    gamma: float = 5.0 / 3.0
    emf_mode: int = 0
    weights: int = 0

    def c(self) -> OrcGrid:
        return OrcGrid(self.nx, self.ny, self.nz, self.dx, self.dy, self.dz,
                       self.gamma, self.emf_mode, self.weights)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


def _state(g: Grid, U, bx, by, bz):
    sh = g.shape
    U = np.ascontiguousarray(U, dtype=np.float64)
    assert U.shape == (8,) + sh, U.shape
    out = [U] + [np.ascontiguousarray(b, dtype=np.float64) for b in (bx, by, bz)]
    for b in out[1:]:
        assert b.shape == sh
    return out


def cell_b(g: Grid, U, bx, by, bz):
    U, bx, by, bz = [a.copy() for a in _state(g, U, bx, by, bz)]
    gc = g.c()
    lib().orc_cell_b(ctypes.byref(gc), _p(bx), _p(by), _p(bz), _p(U))
    return U


def face_fluxes(g: Grid, U, axis: int):
    U = np.ascontiguousarray(U, dtype=np.float64)
    F = np.empty_like(U)
    gc = g.c()
    lib().orc_face_fluxes(ctypes.byref(gc), _p(U), int(axis), _p(F))
    return F


def rhs(g: Grid, U, bx, by, bz):
    """L(U) (8 rows, B rows zero), face rates Lb (3 rows), face fluxes (3x8 rows)."""
    U = cell_b(g, U, bx, by, bz)
    L = np.empty_like(U)
    Lb = np.empty((3,) + g.shape)
    F = np.empty((3, 8) + g.shape)
    gc = g.c()
    lib().orc_rhs(ctypes.byref(gc), _p(U), _p(L), _p(Lb), _p(F[0]), _p(F[1]), _p(F[2]))
    return L, Lb, F


def step(g: Grid, U, bx, by, bz, dt: float, nsteps: int = 1, integrator: str = "ssprk3"):
    """Advance copies of the state by nsteps steps of size dt."""
    U, bx, by, bz = [a.copy() for a in _state(g, U, bx, by, bz)]
    gc = g.c()
    fn = lib().orc_ssprk3_step if integrator == "ssprk3" else lib().orc_rk4_step
    for _ in range(nsteps):
        fn(ctypes.byref(gc), float(dt), _p(U), _p(bx), _p(by), _p(bz))
    return U, bx, by, bz


def step_cfl(g: Grid, U, bx, by, bz, cfl: float, nsteps: int = 1, integrator: str = "ssprk3"):
    """Advance nsteps steps, each with dt = cfl / max speed of its start state."""
    U, bx, by, bz = [a.copy() for a in _state(g, U, bx, by, bz)]
    gc = g.c()
    fn = lib().orc_ssprk3_step if integrator == "ssprk3" else lib().orc_rk4_step
    dts = []
    for _ in range(nsteps):
        lib().orc_cell_b(ctypes.byref(gc), _p(bx), _p(by), _p(bz), _p(U))
        dt = lib().orc_cfl_dt(ctypes.byref(gc), float(cfl), _p(U))
        dts.append(dt)
        fn(ctypes.byref(gc), dt, _p(U), _p(bx), _p(by), _p(bz))
    return U, bx, by, bz, dts


def cfl_speed(g: Grid, U, bx, by, bz) -> float:
    U = cell_b(g, U, bx, by, bz)
    gc = g.c()
    return lib().orc_cfl_speed(ctypes.byref(gc), _p(U))


def cfl_dt(g: Grid, U, bx, by, bz, cfl: float) -> float:
    U = cell_b(g, U, bx, by, bz)
    gc = g.c()
    return lib().orc_cfl_dt(ctypes.byref(gc), float(cfl), _p(U))


def totals(g: Grid, U, bx, by, bz):
    U = cell_b(g, U, bx, by, bz)
    out = np.empty(8)
    gc = g.c()
    lib().orc_totals(ctypes.byref(gc), _p(U), _p(out))
    return out


def div_b(g: Grid, bx, by, bz):
    bx, by, bz = [np.ascontiguousarray(b, dtype=np.float64) for b in (bx, by, bz)]
    out = np.empty(g.shape)
    gc = g.c()
    lib().orc_div_b(ctypes.byref(gc), _p(bx), _p(by), _p(bz), _p(out))
    return out


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> None:
    lib().orc_set_num_threads(int(n))


def library_path() -> str:
    return os.path.abspath(_build.LIB)
