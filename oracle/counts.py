"""Operation counts of the oracle's own steps (test infrastructure).

The same source as the oracle, compiled by ``count_ops.cpp`` with a counting
value type in place of ``double``: add/sub and mul are counted one each
unless an operand is exactly 0 or +-1 (the structural zeros and signs of the
dense eigenvector matrices), div and sqrt separately.  Single-threaded.
Only tests/ and the design notes' figures use it.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import OrcGrid, build as _build

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
KINDS = ("add", "mul", "div", "sqrt")


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(_build.build_count())
        d, i = ctypes.c_double, ctypes.c_int
        G = ctypes.POINTER(OrcGrid)
        L.orc_count_reset.argtypes = []
        L.orc_count_get.argtypes = [ctypes.POINTER(ctypes.c_longlong)]
        L.orc_phi_n.restype = d
        L.orc_phi_n.argtypes = [d, d, d, d]
        L.orc_eigen.restype = i
        L.orc_eigen.argtypes = [_dp, d, _dp, _dp, _dp]
        L.orc_interface_flux_w.argtypes = [_dp, d, i, _dp]
        L.orc_face_fluxes.argtypes = [G, _dp, i, _dp]
        L.orc_ssprk3_step.argtypes = [G, d, _dp, _dp, _dp, _dp]
        L.orc_cfl_dt.restype = d
        L.orc_cfl_dt.argtypes = [G, d, _dp]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def counted(fn, *args):
    """(result, {kind: count}) of one call into the counting build."""
    L = lib()
    L.orc_count_reset()
    r = fn(L, *args)
    out = (ctypes.c_longlong * 4)()
    L.orc_count_get(out)
    return r, dict(zip(KINDS, out[:]))


def phi_n(a, b, c, d):
    return counted(lambda L: L.orc_phi_n(float(a), float(b), float(c), float(d)))


def eigen(W, gamma=5.0 / 3.0):
    W = np.ascontiguousarray(W, dtype=np.float64)
    lam, RU, LU = np.empty(7), np.empty(49), np.empty(49)
    st, n = counted(lambda L: L.orc_eigen(_p(W), gamma, _p(lam), _p(RU), _p(LU)))
    return (lam, RU.reshape(7, 7), LU.reshape(7, 7), st), n


def interface_flux(Us, gamma=5.0 / 3.0, weights=0):
    Us = np.ascontiguousarray(Us, dtype=np.float64).reshape(48)
    F = np.empty(8)
    _, n = counted(lambda L: L.orc_interface_flux_w(_p(Us), gamma, int(weights), _p(F)))
    return F, n


def ssprk3_step(grid: OrcGrid, dt, U, bx, by, bz):
    """One SSP-RK3 step in place (as oracle.ssprk3_step), with its counts."""
    for a in (U, bx, by, bz):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    _, n = counted(lambda L: L.orc_ssprk3_step(ctypes.byref(grid), float(dt), _p(U), _p(bx), _p(by), _p(bz)))
    return n


def cfl_dt(grid: OrcGrid, cfl, U):
    U = np.ascontiguousarray(U, dtype=np.float64)
    return counted(lambda L: L.orc_cfl_dt(ctypes.byref(grid), float(cfl), _p(U)))


def flops(n: dict) -> int:
    """add + mul + div + sqrt (each one flop; the oracle has no FMA)."""
    return sum(n[k] for k in KINDS)
