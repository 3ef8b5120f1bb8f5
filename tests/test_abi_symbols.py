"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/*.h declares; argument validation answers before any CUDA call."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1808_10633_gb300 import build, wombat

    build.build()
    return wombat.load()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(wb_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("wb_init_grid", "wb_step", "wb_cfl_dt", "wb_conserved_totals"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_1808_10633_gb300 import wombat

    assert set(wombat.EXPORTS) == set(declared_functions())


def test_version_string(lib):
    assert b"sm_103a" in lib.wb_version()


def _desc(wombat, **over):
    dims = np.array([8, 8, 8], dtype=np.int32)
    kw = dict(npatch=1, dims=dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), dx=0.1, dy=0.1,
              dz=0.1, gamma=5 / 3, ghost=3, precision=0, integrator=0, emf_mode=0, weights=0)
    kw.update(over)
    return wombat.GridDesc(**kw), dims


@pytest.mark.parametrize("bad", [dict(ghost=2), dict(npatch=0), dict(npatch=1 << 24), dict(dx=0.0), dict(gamma=1.0),
                                 dict(precision=7), dict(integrator=5), dict(emf_mode=3),
                                 dict(weights=2), dict(weights=1, precision=2)])
def test_invalid_descriptor_is_rejected_on_the_host(lib, bad):
    from paper_1808_10633_gb300 import wombat

    d, dims = _desc(wombat, **bad)
    U = np.zeros(8 * 512)
    b = np.zeros(3 * 512)
    h = ctypes.c_void_p()
    rc = lib.wb_init_grid(ctypes.byref(d), U.ctypes.data, b.ctypes.data, None, ctypes.byref(h))
    assert rc == wombat.WB_EINVAL
    assert lib.wb_last_error()


def test_null_arguments_are_rejected(lib):
    from paper_1808_10633_gb300 import wombat

    h = ctypes.c_void_p()
    assert lib.wb_init_grid(None, None, None, None, ctypes.byref(h)) == wombat.WB_EINVAL
    assert lib.wb_step(None, 1e-3, 1) == wombat.WB_EINVAL
    assert lib.wb_step_cfl(None, 0.4, 1) == wombat.WB_EINVAL
    out = ctypes.c_double()
    assert lib.wb_cfl_dt(None, 0.4, ctypes.byref(out)) == wombat.WB_EINVAL
    assert lib.wb_conserved_totals(None, None) == wombat.WB_EINVAL
    assert lib.wb_destroy(None) == wombat.WB_OK


@pytest.mark.parametrize("dims", [(0, 8, 8), (8, -1, 8), (8, 8, 0), (4097, 8, 8), (2048, 2048, 1024)])
def test_empty_or_oversized_patches_are_rejected_on_the_host(lib, dims):
    """A patch with an empty axis, an axis beyond 4096 cells or 2^31 cells or
    more is refused before any device work (WB_EINVAL, message set)."""
    from paper_1808_10633_gb300 import wombat

    d, _ = _desc(wombat)
    arr = np.array(dims, dtype=np.int32)
    d.dims = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    U = np.zeros(8)
    b = np.zeros(3)
    h = ctypes.c_void_p()
    rc = lib.wb_init_grid(ctypes.byref(d), U.ctypes.data, b.ctypes.data, None, ctypes.byref(h))
    assert rc == wombat.WB_EINVAL
    assert b"patch 0" in lib.wb_last_error()
