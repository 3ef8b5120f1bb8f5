"""A periodic world grid cut into linked brick patches (host-side layout).

Sec. 2.2 advances a simulation as patches that are resolved with the ghost
zones of their neighbours.  Here the world of (NX, NY, NZ) cells is cut along
each axis at positions ``cuts = (xc, yc, zc)`` (each list starts at 0 and ends
at the world's extent); brick (a, b, c) covers
``[xc[a], xc[a+1]) x [yc[b], yc[b+1]) x [zc[c], zc[c+1])`` and is patch
``a + nbx * (b + nby * c)`` (x fastest).  The library reads a neighbour's
cells in place through the link table built here, so no ghost zones are
stored or copied.  ``split`` and ``join`` convert between the world arrays
``U[8, NZ, NY, NX]``, ``b[3, NZ, NY, NX]`` and the ABI's patch-major layout.
Nothing here computes on the state.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np


def _check(cuts):
    out = []
    for c in cuts:
        c = [int(v) for v in c]
        assert len(c) >= 2 and c[0] == 0 and all(b > a for a, b in zip(c, c[1:])), c
        out.append(c)
    assert len(out) == 3
    return out


def brick_dims(cuts) -> list:
    xc, yc, zc = _check(cuts)
    return [(xc[a + 1] - xc[a], yc[b + 1] - yc[b], zc[c + 1] - zc[c])
            for c in range(len(zc) - 1) for b in range(len(yc) - 1) for a in range(len(xc) - 1)]


def brick_links(cuts) -> np.ndarray:
    """links[27 p + 9 (oz+1) + 3 (oy+1) + (ox+1)]: the brick that continues
    brick p in direction (ox, oy, oz), periodic round the world."""
    xc, yc, zc = _check(cuts)
    nb = (len(xc) - 1, len(yc) - 1, len(zc) - 1)
    out = np.empty((nb[2], nb[1], nb[0], 27), dtype=np.int32)
    for c in range(nb[2]):
        for b in range(nb[1]):
            for a in range(nb[0]):
                for oz in (-1, 0, 1):
                    for oy in (-1, 0, 1):
                        for ox in (-1, 0, 1):
                            q = ((a + ox) % nb[0]) + nb[0] * (((b + oy) % nb[1]) + nb[1] * ((c + oz) % nb[2]))
                            out[c, b, a, 9 * (oz + 1) + 3 * (oy + 1) + (ox + 1)] = q
    return out.reshape(-1)


def split(U: np.ndarray, b: np.ndarray, cuts: Sequence[Sequence[int]]):
    """World arrays -> flat patch-major arrays (U then b) in brick order."""
    xc, yc, zc = _check(cuts)
    Us, bs = [], []
    for c in range(len(zc) - 1):
        for bb in range(len(yc) - 1):
            for a in range(len(xc) - 1):
                sl = (slice(None), slice(zc[c], zc[c + 1]), slice(yc[bb], yc[bb + 1]), slice(xc[a], xc[a + 1]))
                Us.append(np.ascontiguousarray(U[sl]).ravel())
                bs.append(np.ascontiguousarray(b[sl]).ravel())
    return np.concatenate(Us), np.concatenate(bs)


def join(Uflat: np.ndarray, bflat: np.ndarray, cuts: Sequence[Sequence[int]]):
    """Flat patch-major arrays -> world arrays U[8, NZ, NY, NX], b[3, NZ, NY, NX]."""
    xc, yc, zc = _check(cuts)
    shape = (zc[-1], yc[-1], xc[-1])
    U = np.empty((8,) + shape)
    b = np.empty((3,) + shape)
    oU = ob = 0
    for c in range(len(zc) - 1):
        for bb in range(len(yc) - 1):
            for a in range(len(xc) - 1):
                sh = (zc[c + 1] - zc[c], yc[bb + 1] - yc[bb], xc[a + 1] - xc[a])
                n = sh[0] * sh[1] * sh[2]
                sl = (slice(None), slice(zc[c], zc[c + 1]), slice(yc[bb], yc[bb + 1]), slice(xc[a], xc[a + 1]))
                U[sl] = Uflat[oU:oU + 8 * n].reshape((8,) + sh)
                b[sl] = bflat[ob:ob + 3 * n].reshape((3,) + sh)
                oU += 8 * n
                ob += 3 * n
    return U, b
