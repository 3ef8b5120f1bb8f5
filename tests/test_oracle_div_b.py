"""Pins of the oracle's face divergence of b (orc_div_b), the checker of the
constrained-transport invariant (Sec. 2.1: the staggered-mesh CT keeps the
face divergence of b to round-off).

The checks know the divergence from outside the function:

* gradient of a Fourier mode: with b = grad_h(phi) on the faces (one-sided
  differences of a periodic cell field phi), div_h b is the discrete
  Laplacian of phi, whose eigenvalue on the mode
  cos(2 pi (a i/nx + b j/ny + c k/nz) + theta) is
  -sum_d 4 sin^2(pi m_d/n_d) / dx_d^2 (discrete Fourier analysis);
* the discrete Gauss theorem: over any box of cells, sum(div b) dV equals the
  net outward face flux through the box's boundary faces, for random b;
* a per-cell brute force by faces, written as the outward flux of each
  cell's six faces divided by its volume.

A planted mistake (a dropped axis term, a wrong neighbour, a flipped sign, a
swapped cell size) compiled into a copy of the oracle source must fail at
least one of them.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle as O

SHAPE = (5, 6, 8)            # (nz, ny, nx): every axis its own length
SPACING = (0.13, 0.07, 0.21)  # dx, dy, dz: every axis its own cell size


def _grid():
    nz, ny, nx = SHAPE
    dx, dy, dz = SPACING
    return O.Grid(nx, ny, nz, dx, dy, dz)


def _call(lib, g, bx, by, bz):
    out = np.empty(g.shape)
    gc = g.c()
    dp = ctypes.POINTER(ctypes.c_double)
    p = lambda a: a.ctypes.data_as(dp)
    lib.orc_div_b(ctypes.byref(gc), p(bx), p(by), p(bz), p(out))
    return out


def _fourier_error(div_fn):
    """Largest error of div_h(grad_h phi) against the closed-form eigenvalue,
    relative to max|b|/dx, over several modes."""
    g = _grid()
    nz, ny, nx = SHAPE
    dx, dy, dz = SPACING
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    worst = 0.0
    for (a, b, c, th) in [(1, 0, 0, 0.3), (0, 2, 0, 1.1), (0, 0, 1, -0.4), (1, 1, 2, 0.7), (3, -2, 1, 2.0)]:
        phi = np.cos(2 * np.pi * (a * i / nx + b * j / ny + c * k / nz) + th)
        bx = np.ascontiguousarray((phi - np.roll(phi, 1, axis=2)) / dx)
        by = np.ascontiguousarray((phi - np.roll(phi, 1, axis=1)) / dy)
        bz = np.ascontiguousarray((phi - np.roll(phi, 1, axis=0)) / dz)
        lam = -(4 * np.sin(np.pi * a / nx) ** 2 / dx ** 2 + 4 * np.sin(np.pi * b / ny) ** 2 / dy ** 2
                + 4 * np.sin(np.pi * c / nz) ** 2 / dz ** 2)
        got = div_fn(g, bx, by, bz)
        scale = max(np.abs(bx).max() / dx, np.abs(by).max() / dy, np.abs(bz).max() / dz)
        worst = max(worst, np.abs(got - lam * phi).max() / scale)
    return worst


def _gauss_error(div_fn, seed=5):
    """Largest error of sum_box(div) dV against the net face flux out of the
    box, relative to the sum of |flux| over the box's faces, for random b and
    random boxes (boxes may reach the upper edge, whose faces wrap)."""
    rng = np.random.default_rng(seed)
    g = _grid()
    nz, ny, nx = SHAPE
    dx, dy, dz = SPACING
    bx, by, bz = [np.ascontiguousarray(rng.standard_normal(SHAPE)) for _ in range(3)]
    div = div_fn(g, bx, by, bz)
    worst = 0.0
    for _ in range(40):
        i0, j0, k0 = (int(rng.integers(0, n)) for n in (nx, ny, nz))
        i1, j1, k1 = (int(rng.integers(s + 1, n + 1)) for s, n in ((i0, nx), (j0, ny), (k0, nz)))
        vol = dx * dy * dz * div[k0:k1, j0:j1, i0:i1].sum()
        ax, ay, az = dy * dz, dx * dz, dx * dy
        fx = (bx[k0:k1, j0:j1, i1 % nx] - bx[k0:k1, j0:j1, i0]) * ax
        fy = (by[k0:k1, j1 % ny, i0:i1] - by[k0:k1, j0, i0:i1]) * ay
        fz = (bz[k1 % nz, j0:j1, i0:i1] - bz[k0, j0:j1, i0:i1]) * az
        flux = fx.sum() + fy.sum() + fz.sum()
        mag = np.abs(fx).sum() + np.abs(fy).sum() + np.abs(fz).sum()
        worst = max(worst, abs(vol - flux) / mag)
    return worst


def _cell_error(div_fn, seed=6):
    """Largest error against the outward flux of each cell's six faces over
    its volume, cell by cell in plain loops."""
    rng = np.random.default_rng(seed)
    g = _grid()
    nz, ny, nx = SHAPE
    dx, dy, dz = SPACING
    bx, by, bz = [np.ascontiguousarray(rng.standard_normal(SHAPE)) for _ in range(3)]
    div = div_fn(g, bx, by, bz)
    worst = 0.0
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                out = ((bx[k, j, (i + 1) % nx] - bx[k, j, i]) * dy * dz
                       + (by[k, (j + 1) % ny, i] - by[k, j, i]) * dx * dz
                       + (bz[(k + 1) % nz, j, i] - bz[k, j, i]) * dx * dy)
                worst = max(worst, abs(div[k, j, i] - out / (dx * dy * dz)) * min(SPACING))
    return worst


def test_div_b_of_a_face_gradient_is_the_discrete_laplacian(orc):
    assert _fourier_error(orc.div_b) <= 1e-14


def test_div_b_obeys_the_discrete_gauss_theorem(orc):
    assert _gauss_error(orc.div_b) <= 1e-14


def test_div_b_is_the_outward_face_flux_per_volume(orc):
    assert _cell_error(orc.div_b) <= 1e-14


# Planted mistakes, each a text edit of orc_div_b's body in a copy of the
# oracle source (compiled on the CPU into the test's temporary folder).
MUTANTS = {
    "drop the z term": ("+ (bz[IDX(g, i, j, wrapi(k + 1, g->nz))] - bz[c]) / g->dz", "+ 0.0"),
    "wrong x neighbour": ("bx[IDX(g, wrapi(i + 1, g->nx), j, k)]", "bx[IDX(g, wrapi(i - 1, g->nx), j, k)]"),
    "flipped y sign": ("(by[IDX(g, i, wrapi(j + 1, g->ny), k)] - by[c])",
                       "(by[c] - by[IDX(g, i, wrapi(j + 1, g->ny), k)])"),
    "dx for dy": ("- by[c]) / g->dy", "- by[c]) / g->dx"),
    "y neighbour along x": ("by[IDX(g, i, wrapi(j + 1, g->ny), k)]", "by[IDX(g, wrapi(i + 1, g->nx), j, k)]"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_div_b_mistake_is_caught(tmp_path, name):
    with open(os.path.join(os.path.dirname(O.__file__), "wb_oracle.c")) as f:
        src = f.read()
    head = src.index("void orc_div_b(")
    body = src[head:]
    old, new = MUTANTS[name]
    assert body.count(old) == 1, name
    mutant = src[:head] + body.replace(old, new)
    path = tmp_path / "wb_oracle.c"
    path.write_text(mutant)
    lib = tmp_path / "libmutant.so"
    inc = os.path.dirname(O.__file__)
    subprocess.run([os.environ.get("CC", "gcc"), "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                    "-I", inc, str(path), "-o", str(lib), "-lm"], check=True)
    L = ctypes.CDLL(str(lib))
    L.orc_div_b.argtypes = [ctypes.POINTER(O.OrcGrid)] + [ctypes.POINTER(ctypes.c_double)] * 4
    fn = lambda g, bx, by, bz: _call(L, g, bx, by, bz)
    errs = (_fourier_error(fn), _gauss_error(fn), _cell_error(fn))
    assert max(errs) > 1e-6, (name, errs)
