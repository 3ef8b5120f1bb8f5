"""Host side of linked brick patches: the world <-> patch layout round trip,
and the library's link-table checks, which answer before any CUDA call."""
import ctypes

import numpy as np
import pytest

from paper_1808_10633_gb300 import bricks

CUTS = ([0, 5, 12, 20], [0, 7, 16], [0, 3, 9])


@pytest.fixture(scope="module")
def wombat():
    from paper_1808_10633_gb300 import build, wombat

    build.build()
    wombat.load()
    return wombat


def test_split_join_round_trip():
    rng = np.random.default_rng(0)
    U = rng.standard_normal((8, 9, 16, 20))
    b = rng.standard_normal((3, 9, 16, 20))
    Uf, bf = bricks.split(U, b, CUTS)
    dims = bricks.brick_dims(CUTS)
    assert Uf.size == 8 * sum(x * y * z for x, y, z in dims)
    # first brick comes first, x fastest inside it
    assert np.array_equal(Uf[:5 * 7 * 3 * 8].reshape(8, 3, 7, 5), U[:, :3, :7, :5])
    U2, b2 = bricks.join(Uf, bf, CUTS)
    assert np.array_equal(U2, U) and np.array_equal(b2, b)


def test_links_are_periodic_neighbours():
    L = bricks.brick_links(CUTS).reshape(-1, 27)
    nb = (3, 2, 2)
    for p in range(L.shape[0]):
        a, r = p % 3, p // 3
        b_, c = r % 2, r // 2
        assert L[p, 13] == p
        assert L[p, 14] == (a + 1) % 3 + 3 * (b_ + 2 * c)          # +x
        assert L[p, 12] == (a - 1) % 3 + 3 * (b_ + 2 * c)          # -x
        assert L[p, 16] == a + 3 * ((b_ + 1) % 2 + 2 * c)          # +y
        assert L[p, 22] == a + 3 * (b_ + 2 * ((c + 1) % 2))        # +z
        assert L[p, 0] == (a - 1) % 3 + 3 * ((b_ - 1) % 2 + 2 * ((c - 1) % 2))


def _init(wombat, dims, links):
    flat = np.array([v for d in dims for v in d], dtype=np.int32)
    lk = np.ascontiguousarray(links, dtype=np.int32)
    desc = wombat.GridDesc(len(dims), flat.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), 0.1, 0.1,
                           0.1, 5 / 3, 3, 0, 0, 0, 0, lk.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    n = sum(x * y * z for x, y, z in dims)
    U = np.ones(8 * n)
    b = np.zeros(3 * n)
    h = ctypes.c_void_p()
    rc = wombat.load().wb_init_grid(ctypes.byref(desc), U.ctypes.data, b.ctypes.data, None, ctypes.byref(h))
    if rc == wombat.WB_OK:
        wombat.load().wb_destroy(h)
    return rc


def test_valid_links_pass_the_checks(wombat):
    rc = _init(wombat, bricks.brick_dims(CUTS), bricks.brick_links(CUTS))
    # without a GPU the call stops at the first CUDA call, after the checks
    assert rc in (wombat.WB_OK, wombat.WB_ECUDA), wombat.load().wb_last_error()


def test_self_links_on_a_thin_axis_pass(wombat):
    cuts = ([0, 8, 20], [0, 6, 16], [0, 1])
    rc = _init(wombat, bricks.brick_dims(cuts), bricks.brick_links(cuts))
    assert rc in (wombat.WB_OK, wombat.WB_ECUDA), wombat.load().wb_last_error()


@pytest.mark.parametrize("case", ["range", "centre", "reciprocal", "diagonal", "extent", "thin"])
def test_broken_links_are_rejected(wombat, case):
    dims = bricks.brick_dims(CUTS)
    L = bricks.brick_links(CUTS).reshape(-1, 27).copy()
    if case == "range":
        L[3, 5] = len(dims)
    elif case == "centre":
        L[2, 13] = 0
    elif case == "reciprocal":
        L[0, 14], L[0, 12] = L[0, 12], L[0, 14]
    elif case == "diagonal":
        L[4, 0] = L[4, 1]
    elif case == "extent":
        dims = [tuple(d) for d in dims]
        dims[1] = (dims[1][0], dims[1][1] + 1, dims[1][2])
    elif case == "thin":
        cuts = ([0, 2, 12, 20], [0, 7, 16], [0, 3, 9])
        dims = bricks.brick_dims(cuts)
        L = bricks.brick_links(cuts).reshape(-1, 27)
    rc = _init(wombat, dims, L)
    assert rc == wombat.WB_EINVAL, (case, rc)
    assert b"links" in wombat.load().wb_last_error()
