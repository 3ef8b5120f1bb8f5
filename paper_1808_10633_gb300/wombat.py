"""Thin ctypes binding of libwombat_gb300.so (include/wombat_gb300.h).

Argument marshalling only: every step of the method runs in the CUDA
library.  There is no CPU fallback; loading fails loudly when the library is
missing.  Host arrays are numpy float64 arrays (pageable) or pinned torch
tensors; the CUDA stream handle may come from torch.cuda.current_stream().
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# WB_LIBRARY selects another build of the library (e.g. the bounds-checked one)
LIB_PATH = os.environ.get("WB_LIBRARY") or os.path.join(HERE, "libwombat_gb300.so")

WB_OK, WB_EINVAL, WB_ECUDA, WB_ENOMEM, WB_ENONFINITE, WB_ETIMEOUT, WB_EINTERNAL = 0, -1, -2, -3, -4, -5, -6
WB_FP64, WB_FP32, WB_FP32_LEARNED = 0, 1, 2
WB_SSPRK3, WB_RK4 = 0, 1
PRECISIONS = {"fp64": WB_FP64, "fp32": WB_FP32, "learned": WB_FP32_LEARNED}
INTEGRATORS = {"ssprk3": WB_SSPRK3, "rk4": WB_RK4}

# every entry point declared in include/wombat_gb300.h
EXPORTS = ("wb_init_grid", "wb_set_state", "wb_step", "wb_step_cfl", "wb_cfl_dt",
           "wb_conserved_totals", "wb_get_state", "wb_sync", "wb_get_info", "wb_destroy",
           "wb_last_error", "wb_version", "wb_step_profiled", "wb_alu_peak", "wb_face_fluxes",
           "wb_conserved_totals_noalloc", "wb_mlp_loss_grad", "wb_mlp_train", "wb_harvest", "wb_cell_state_flux", "wb_set_mlp", "wb_set_mlp_gate", "wb_autotune", "wb_set_tiles",
           "wb_learned_stats", "wb_div_b", "wb_set_step_totals", "wb_step_totals",
           "wb_set_state_f32", "wb_get_state_f32")
MLP_NFIELD, MLP_NPARAM, MLP_RECORD = 7, 1379, 12
TILE_CANDIDATES = ("per-patch model", "shape 0", "shape 1", "shape 2", "per-patch model by shape")
KERNEL_CLASSES = ("sweep_x", "sweep_y", "sweep_z", "update", "cfl", "dt", "totals", "emf")


class WombatError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"wombat error {code}: {msg}")
        self.code = code


class GridDesc(ctypes.Structure):
    _fields_ = [
        ("npatch", ctypes.c_int), ("dims", ctypes.POINTER(ctypes.c_int)),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
        ("gamma", ctypes.c_double), ("ghost", ctypes.c_int), ("precision", ctypes.c_int),
        ("integrator", ctypes.c_int), ("emf_mode", ctypes.c_int), ("weights", ctypes.c_int),
        ("links", ctypes.POINTER(ctypes.c_int)),
    ]


class GridInfo(ctypes.Structure):
    _fields_ = [
        ("npatch", ctypes.c_int), ("ncells", ctypes.c_longlong), ("precision", ctypes.c_int),
        ("integrator", ctypes.c_int), ("emf_mode", ctypes.c_int),
        ("device_bytes", ctypes.c_longlong), ("time", ctypes.c_double), ("steps", ctypes.c_longlong),
    ]


_lib = None


def load() -> ctypes.CDLL:
    """Load the in-tree library (built by __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                          "(there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    vp, dp, i, d = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_double
    L.wb_init_grid.argtypes = [ctypes.POINTER(GridDesc), vp, vp, vp, ctypes.POINTER(vp)]
    L.wb_set_state.argtypes = [vp, vp, vp]
    L.wb_step.argtypes = [vp, d, i]
    L.wb_step_cfl.argtypes = [vp, d, i]
    L.wb_cfl_dt.argtypes = [vp, d, dp]
    L.wb_conserved_totals.argtypes = [vp, dp]
    L.wb_get_state.argtypes = [vp, vp, vp]
    L.wb_sync.argtypes = [vp]
    L.wb_get_info.argtypes = [vp, ctypes.POINTER(GridInfo)]
    L.wb_destroy.argtypes = [vp]
    L.wb_step_profiled.argtypes = [vp, d, i, i, dp, ctypes.POINTER(ctypes.c_int), dp]
    L.wb_alu_peak.argtypes = [i, dp]
    L.wb_face_fluxes.argtypes = [vp, i, vp]
    L.wb_conserved_totals_noalloc.argtypes = [vp, i, ctypes.c_longlong, d, vp, vp]
    L.wb_set_mlp.argtypes = [vp, vp, d, d]
    L.wb_set_mlp_gate.argtypes = [vp, d]
    L.wb_autotune.argtypes = [vp, vp]
    L.wb_set_tiles.argtypes = [vp, ctypes.c_int]
    L.wb_learned_stats.argtypes = [vp, vp, i]
    L.wb_div_b.argtypes = [vp, dp]
    L.wb_set_step_totals.argtypes = [vp, i]
    L.wb_set_state_f32.argtypes = [vp, vp, vp]
    L.wb_get_state_f32.argtypes = [vp, vp, vp]
    L.wb_step_totals.argtypes = [vp, dp]
    L.wb_harvest.argtypes = [vp, i, vp, ctypes.c_longlong, vp, vp, d, d, vp]
    L.wb_cell_state_flux.argtypes = [vp, i, vp, vp]
    L.wb_mlp_loss_grad.argtypes = [vp, ctypes.c_longlong, vp, d, vp, vp]
    L.wb_mlp_train.argtypes = [vp, ctypes.c_longlong, vp, i, i, d, d, ctypes.c_ulonglong, vp]
    L.wb_last_error.restype = ctypes.c_char_p
    L.wb_version.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("wb_last_error", "wb_version"):
            getattr(L, name).restype = i
    _lib = L
    return L


def _check(rc: int):
    if rc != WB_OK:
        raise WombatError(rc, load().wb_last_error().decode())


def _ptr(a, fp32: bool = False) -> int:
    """Host pointer of a C-contiguous float64 (fp32: float32) numpy array or
    pinned torch tensor."""
    if isinstance(a, np.ndarray):
        want = np.float32 if fp32 else np.float64
        assert a.dtype == want and a.flags.c_contiguous, f"need C-contiguous {np.dtype(want).name}"
        return a.ctypes.data
    want = "torch.float32" if fp32 else "torch.float64"
    assert str(a.dtype) == want and a.is_contiguous() and not a.is_cuda, f"need a host {want} tensor"
    return a.data_ptr()


def _is_fp32(a) -> bool:
    return str(getattr(a, "dtype", "")) in ("float32", "torch.float32")


class Grid:
    """A set of periodic patches advanced by the CUDA library.

    U: (npatch*8*cells) or (8, nz, ny, nx) float64 host array in the ABI
    layout; b: faces (3, nz, ny, nx) or flat.  dims: list of (nx, ny, nz)."""

    def __init__(self, dims: Sequence[Sequence[int]], dx, dy, dz, U, b, gamma=5.0 / 3.0,
                 precision="fp64", integrator="ssprk3", emf_mode=0, stream=None, weights="js",
                 links=None):
        L = load()
        self._lib = L
        self.dims = [tuple(int(v) for v in d) for d in dims]
        self.ncells = sum(d[0] * d[1] * d[2] for d in self.dims)
        flat = np.array([v for d in self.dims for v in d], dtype=np.int32)
        self._dims = flat
        lk = None
        if links is not None:
            lk = np.ascontiguousarray(links, dtype=np.int32).ravel()
            assert lk.size == 27 * len(self.dims), (lk.size, len(self.dims))
        self._links = lk
        desc = GridDesc(len(self.dims), flat.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                        float(dx), float(dy), float(dz), float(gamma), 3,
                        PRECISIONS.get(precision, precision) if isinstance(precision, str) else precision,
                        INTEGRATORS.get(integrator, integrator) if isinstance(integrator, str) else integrator,
                        int(emf_mode), {"js": 0, "z": 1}.get(weights, weights),
                        lk.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) if lk is not None else None)
        self.precision = precision
        U = self._host(U, 8)
        b = self._host(b, 3)
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(int(stream)) if stream else None
        _check(L.wb_init_grid(ctypes.byref(desc), _ptr(U), _ptr(b), st, ctypes.byref(h)))
        self._h = h

    def _host(self, a, nf, dtype=np.float64):
        if isinstance(a, np.ndarray):
            a = np.ascontiguousarray(a, dtype=dtype)
            assert a.size == nf * self.ncells, (a.shape, nf, self.ncells)
        return a

    @classmethod
    def from_bricks(cls, st, cuts, **kw):
        """The world state `st` split at `cuts` (x, y, z cut positions, each
        starting at 0 and ending at the world's extent) into linked brick
        patches (see bricks.py)."""
        from . import bricks

        U, b = bricks.split(st.U, np.stack([st.bx, st.by, st.bz]), cuts)
        return cls(bricks.brick_dims(cuts), st.dx, st.dy, st.dz, U, b, gamma=st.gamma,
                   links=bricks.brick_links(cuts), **kw)

    @classmethod
    def from_state(cls, st, **kw):
        nx, ny, nz = st.dims
        b = np.stack([st.bx, st.by, st.bz])
        return cls([(nx, ny, nz)], st.dx, st.dy, st.dz, st.U, b, gamma=st.gamma, **kw)

    @classmethod
    def from_patches(cls, states, **kw):
        dims = [s.dims for s in states]
        U = np.concatenate([s.U.ravel() for s in states])
        b = np.concatenate([np.stack([s.bx, s.by, s.bz]).ravel() for s in states])
        s0 = states[0]
        return cls(dims, s0.dx, s0.dy, s0.dz, U, b, gamma=s0.gamma, **kw)

    # -- calls -------------------------------------------------------------
    def set_state(self, U, b):
        """Replace the state; float32 arrays (FP32 grids) take the FP32 entry point."""
        if _is_fp32(U) and _is_fp32(b):
            _check(self._lib.wb_set_state_f32(self._h, _ptr(self._host(U, 8, np.float32), True),
                                              _ptr(self._host(b, 3, np.float32), True)))
        else:
            _check(self._lib.wb_set_state(self._h, _ptr(self._host(U, 8)), _ptr(self._host(b, 3))))

    def step(self, dt: float, nsteps: int = 1):
        _check(self._lib.wb_step(self._h, float(dt), int(nsteps)))

    def step_cfl(self, cfl: float = 0.4, nsteps: int = 1):
        _check(self._lib.wb_step_cfl(self._h, float(cfl), int(nsteps)))

    def step_profiled(self, cfl: float, nsteps: int, with_totals: bool = True):
        """CFL steps with per-kernel CUDA-event timing on the grid's stream.
        Returns (total_ms, {class: ms}, {class: launches})."""
        ms = (ctypes.c_double * len(KERNEL_CLASSES))()
        cnt = (ctypes.c_int * len(KERNEL_CLASSES))()
        tot = ctypes.c_double()
        _check(self._lib.wb_step_profiled(self._h, float(cfl), int(nsteps), int(bool(with_totals)),
                                          ms, cnt, ctypes.byref(tot)))
        return (tot.value, dict(zip(KERNEL_CLASSES, ms[:])), dict(zip(KERNEL_CLASSES, cnt[:])))

    def cfl_dt(self, cfl: float = 0.4) -> float:
        out = ctypes.c_double()
        _check(self._lib.wb_cfl_dt(self._h, float(cfl), ctypes.byref(out)))
        return out.value

    def totals(self) -> np.ndarray:
        out = (ctypes.c_double * 8)()
        _check(self._lib.wb_conserved_totals(self._h, out))
        return np.array(out[:])

    def set_step_totals(self, on: bool = True):
        """Take the conserved totals of every step's start state, overlapped
        with the step's first stages."""
        _check(self._lib.wb_set_step_totals(self._h, int(bool(on))))

    def step_totals(self) -> np.ndarray:
        """Totals of the start state of the last step taken."""
        out = (ctypes.c_double * 8)()
        _check(self._lib.wb_step_totals(self._h, out))
        return np.array(out[:])

    def div_b(self):
        """(max |face divergence of b|, max |b| over faces), FP64."""
        out = (ctypes.c_double * 2)()
        _check(self._lib.wb_div_b(self._h, out))
        return float(out[0]), float(out[1])

    def get_state(self, U_out=None, b_out=None, dtype=np.float64):
        """Returns (U, b) as flat float64 (or float32) arrays, or fills the
        given buffers; float32 buffers take the FP32 entry point."""
        U = np.empty(8 * self.ncells, dtype=dtype) if U_out is None else U_out
        b = np.empty(3 * self.ncells, dtype=dtype) if b_out is None else b_out
        if _is_fp32(U) and _is_fp32(b):
            _check(self._lib.wb_get_state_f32(self._h, _ptr(U, True), _ptr(b, True)))
        else:
            _check(self._lib.wb_get_state(self._h, _ptr(U), _ptr(b)))
        return U, b

    def get_state_single(self):
        """(U[8,nz,ny,nx], bx, by, bz) for a one-patch grid."""
        nx, ny, nz = self.dims[0]
        U, b = self.get_state()
        b = b.reshape(3, nz, ny, nx)
        return U.reshape(8, nz, ny, nx), b[0], b[1], b[2]

    def face_fluxes(self, axis: int) -> np.ndarray:
        """Numerical fluxes of one sweep on the current state, (7, ncells)."""
        out = np.empty(7 * self.ncells)
        _check(self._lib.wb_face_fluxes(self._h, int(axis), out.ctypes.data))
        return out.reshape(7, self.ncells)

    def autotune(self) -> np.ndarray:
        """Measure and keep the fastest sweep tile tables; times (3, 5) in ms
        per axis for TILE_CANDIDATES (per-patch model, shape 0, shape 1,
        shape 2, per-patch model ordered by shape)."""
        ms = np.empty(3 * len(TILE_CANDIDATES))
        _check(self._lib.wb_autotune(self._h, ms.ctypes.data))
        return ms.reshape(3, len(TILE_CANDIDATES))

    def set_tiles(self, candidate: int):
        """Install one of the autotuner's tile tables (an index into
        TILE_CANDIDATES) without timing it."""
        _check(self._lib.wb_set_tiles(self._h, int(candidate)))

    def set_mlp(self, params, kappa: float = 4.0, pjump: float = 0.5, smooth: float | None = None):
        """Install the learned-weight networks (7 x 1379 floats); `smooth`
        sets the smoothness gate (wb_set_mlp_gate) as well."""
        p = np.ascontiguousarray(params, dtype=np.float32).reshape(MLP_NFIELD * MLP_NPARAM)
        _check(self._lib.wb_set_mlp(self._h, p.ctypes.data, float(kappa), float(pjump)))
        if smooth is not None:
            self.set_mlp_gate(smooth)

    def set_mlp_gate(self, smooth: float):
        """Use the networks only where the smoothness indicators spread by
        more than the ratio `smooth` (0: wherever no detector fires)."""
        _check(self._lib.wb_set_mlp_gate(self._h, float(smooth)))

    def learned_stats(self, reset: bool = False):
        """(decisions that kept the Jiang-Shu weights, all weight decisions)
        counted by the learned sweeps."""
        out = (ctypes.c_longlong * 2)()
        _check(self._lib.wb_learned_stats(self._h, out, int(bool(reset))))
        return int(out[0]), int(out[1])

    def harvest(self, axis: int, cells, hU, hF, kappa: float = 4.0, pjump: float = 0.5):
        """Training records (n, 14, 12) for the lower faces of `cells` along axis."""
        c = np.ascontiguousarray(cells, dtype=np.int64)
        hu = np.ascontiguousarray(hU, dtype=np.float64).reshape(-1, 7)
        hf = np.ascontiguousarray(hF, dtype=np.float64).reshape(-1, 7)
        assert hu.shape[0] == c.size == hf.shape[0]
        out = np.empty((c.size, 14, MLP_RECORD), dtype=np.float32)
        _check(self._lib.wb_harvest(self._h, int(axis), c.ctypes.data, c.size, hu.ctypes.data,
                                    hf.ctypes.data, float(kappa), float(pjump), out.ctypes.data))
        return out

    def cell_state_flux(self, axis: int):
        """(X, F), each (7, nz, ny, nx): the rotated conservative 7-vector of
        every cell of patch 0 and its physical flux along `axis`."""
        nx, ny, nz = self.dims[0]
        X = np.empty((7, nz, ny, nx))
        F = np.empty((7, nz, ny, nx))
        _check(self._lib.wb_cell_state_flux(self._h, int(axis), X.ctypes.data, F.ctypes.data))
        return X, F

    def sync(self):
        _check(self._lib.wb_sync(self._h))

    def info(self) -> dict:
        inf = GridInfo()
        _check(self._lib.wb_get_info(self._h, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in GridInfo._fields_}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.wb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def conserved_totals_noalloc(state_ptr: int, precision, ncells: int, dV: float, out_ptr: int,
                             stream=None):
    """Totals of a caller-owned device state (device pointers), no allocation.
    See wb_conserved_totals_noalloc in include/wombat_gb300.h."""
    p = PRECISIONS.get(precision, precision) if isinstance(precision, str) else precision
    _check(load().wb_conserved_totals_noalloc(ctypes.c_void_p(state_ptr), int(p), int(ncells),
                                              float(dV), ctypes.c_void_p(out_ptr),
                                              ctypes.c_void_p(int(stream)) if stream else None))


def mlp_loss_grad(records: np.ndarray, params: np.ndarray, lam: float):
    """GPU loss per field and gradient (7, 1379) of the learned-weight networks."""
    rec = np.ascontiguousarray(records, dtype=np.float32).reshape(-1, MLP_RECORD)
    p = np.ascontiguousarray(params, dtype=np.float32).reshape(MLP_NFIELD * MLP_NPARAM)
    loss = np.empty(MLP_NFIELD)
    grad = np.empty(MLP_NFIELD * MLP_NPARAM, dtype=np.float32)
    _check(load().wb_mlp_loss_grad(rec.ctypes.data, rec.shape[0], p.ctypes.data, float(lam),
                                   loss.ctypes.data, grad.ctypes.data))
    return loss, grad.reshape(MLP_NFIELD, MLP_NPARAM)


def mlp_train(records: np.ndarray, params: np.ndarray, steps: int, batch: int = 4096,
              lr: float = 1e-3, lam: float = 1e-3, seed: int = 1808):
    """Adam training on the GPU; returns (params, loss history (steps, 7))."""
    rec = np.ascontiguousarray(records, dtype=np.float32).reshape(-1, MLP_RECORD)
    p = np.array(params, dtype=np.float32).reshape(MLP_NFIELD * MLP_NPARAM).copy()
    hist = np.empty((max(steps, 1), MLP_NFIELD), dtype=np.float32)
    _check(load().wb_mlp_train(rec.ctypes.data, rec.shape[0], p.ctypes.data, int(steps), int(batch),
                               float(lr), float(lam), int(seed), hist.ctypes.data))
    return p.reshape(MLP_NFIELD, MLP_NPARAM), hist[:steps]


def version() -> str:
    return load().wb_version().decode()


def alu_peak_tflops(precision="fp32") -> float:
    """Measured FMA throughput of the current GPU (TFLOP/s)."""
    out = ctypes.c_double()
    p = PRECISIONS.get(precision, precision) if isinstance(precision, str) else precision
    _check(load().wb_alu_peak(p, ctypes.byref(out)))
    return out.value
