"""Learned WENO weights: training pipeline (data from the solver's own
states, training with the library's CUDA kernels).

1. Targets.  The flux of eq. FWENO at face i+1/2 is the value there of the
   function h whose cell average over cell i is the point value F_i (finite
   differences in the Shu-Osher form).  On a periodic grid h follows from F
   exactly in Fourier space (h^(k) = F^(k) (theta/2)/sin(theta/2), theta =
   2 pi k / N, shifted by half a cell): `face_reconstruction`.  This is exact
   for band-limited data such as the seeded turbulence states.
2. Records.  `harvest` takes each cell's rotated state and physical flux
   from the library (wb_cell_state_flux), reconstructs their face values,
   samples faces and lets the library (wb_harvest) project stencils and
   targets on the interface eigenvectors, split them, normalise them and
   flag detector hits.
3. Training.  `train` runs the library's forward/backward/Adam kernels
   (wb_mlp_train) on the unflagged records.

Parameters are float32 arrays (7, 1379); the layout is in the public header.
"""
from __future__ import annotations

import numpy as np

from . import wombat

D_LIN = np.array([0.1, 0.6, 0.3])
NH, NIN, NOUT = 32, 6, 3


def face_reconstruction(f, npaxis):
    """Exact face values h_{i+1/2} (upper face of cell i) along numpy axis
    `npaxis` of periodic point values f whose cell averages h reproduce."""
    g = np.moveaxis(f, npaxis, -1)
    N = g.shape[-1]
    k = np.arange(N // 2 + 1)
    th = 2.0 * np.pi * k / N
    with np.errstate(divide="ignore", invalid="ignore"):
        fac = np.where(th == 0.0, 1.0, (th / 2.0) / np.sin(th / 2.0))
    fac = fac * np.exp(0.5j * th)
    if N % 2 == 0:
        fac[-1] = 0.0            # Nyquist mode: no real half-cell shift
    h = np.fft.irfft(np.fft.rfft(g, axis=-1) * fac, n=N, axis=-1)
    return np.moveaxis(h, -1, npaxis)


def harvest(st, nsamples: int, seed: int = 1808, kappa: float = 4.0, pjump: float = 0.5,
            axes=(0, 1, 2)):
    """Records (m, 12) from nsamples random faces per axis of state `st`
    (an inputs.State), computed by the library on an FP64 grid."""
    rng = np.random.default_rng(seed)
    g = wombat.Grid.from_state(st, precision="fp64")
    nx, ny, nz = st.dims
    out = []
    for axis in axes:
        X, F = g.cell_state_flux(axis)
        npax = {0: -1, 1: -2, 2: -3}[axis]
        hX = face_reconstruction(X, npax)
        hF = face_reconstruction(F, npax)
        idx = rng.integers(0, [nx, ny, nz], size=(nsamples, 3))
        cells = (idx[:, 2] * ny + idx[:, 1]) * nx + idx[:, 0]
        low = idx.copy()                                  # lower face of cell = upper face of cell - e
        low[:, axis] = (low[:, axis] - 1) % (nx, ny, nz)[axis]
        hu = hX[:, low[:, 2], low[:, 1], low[:, 0]].T
        hf = hF[:, low[:, 2], low[:, 1], low[:, 0]].T
        out.append(g.harvest(axis, cells, hu, hf, kappa, pjump).reshape(-1, wombat.MLP_RECORD))
    g.close()
    return np.concatenate(out)


def init_params(seed: int = 1808):
    """Small random hidden layers and an output layer that starts at the
    linear weights (W3 = 0, b3 = log d)."""
    rng = np.random.default_rng(seed)
    P = []
    for _ in range(wombat.MLP_NFIELD):
        W1 = rng.standard_normal((NH, NIN)) * np.sqrt(1.0 / NIN)
        W2 = rng.standard_normal((NH, NH)) * np.sqrt(1.0 / NH)
        W3 = np.zeros((NOUT, NH))
        P.append(np.concatenate([W1.ravel(), np.zeros(NH), W2.ravel(), np.zeros(NH), W3.ravel(),
                                 np.log(D_LIN)]))
    return np.array(P, dtype=np.float32)


def train(records, params=None, steps: int = 2000, batch: int = 4096, lr: float = 2e-3,
          lam: float = 1e-3, seed: int = 1808):
    """Adam on the GPU; returns (params (7, 1379), loss history (steps, 7))."""
    if params is None:
        params = init_params(seed)
    return wombat.mlp_train(records, params, steps, batch, lr, lam, seed)


def alfven_gain(params, Ns=(16, 32, 64), T: float = 0.2, kappa: float = 4.0, pjump: float = 0.5,
                smooth: float | None = None):
    """What the networks gain: the L1 error of B_y against the exact
    travelling solution of the circularly polarised Alfven wave (amplitude
    0.1, along x, N x 1 x 1 cells) at time T, for the learned weights and,
    on FP32 grids of the same resolution, the Jiang-Shu and WENO-Z weights.
    Returns {N: {"learned", "js", "weno_z", "vs_js", "vs_weno_z",
    "js_decisions"}} (js_decisions: fraction of weight decisions that kept
    the Jiang-Shu weights)."""
    from . import inputs

    out = {}
    for N in Ns:
        errs = {}
        for name, prec, weights in (("learned", "learned", "js"), ("js", "fp32", "js"), ("weno_z", "fp32", "z")):
            st = inputs.alfven_wave(N, 1, 1, amp=0.1)
            g = wombat.Grid.from_state(st, precision=prec, weights=weights)
            if prec == "learned":
                g.set_mlp(params, kappa, pjump, smooth=smooth)
            n = int(np.ceil(T / (0.4 / (3 * 1.2 * N))))
            g.step(T / n, n)
            U = g.get_state_single()[0]
            if prec == "learned":
                fired, dec = g.learned_stats()
                errs["js_decisions"] = fired / max(dec, 1)
            g.close()
            ex = inputs.alfven_wave(N, 1, 1, amp=0.1, t=T)
            errs[name] = float(np.abs(U[5] - ex.U[5]).mean())
        errs["vs_js"] = errs["learned"] / errs["js"]
        errs["vs_weno_z"] = errs["learned"] / errs["weno_z"]
        out[N] = errs
    return out
