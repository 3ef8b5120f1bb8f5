"""Parity cases re-run on the bounds-checked build of the library.

The "check" variant tests every global and shared index the solver kernels
form against its array; an index outside sets a status bit that every
synchronising call reports as WB_EINTERNAL (the access is redirected to an
in-range element instead).  The GPU parity suites (ragged tiles, thin axes,
patches of every tile shape, autotuned tables, WENO-Z, RK4, both EMF modes,
linked bricks, the learned sweep) pass on it unchanged, so none of those
launches formed an out-of-range index."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_suites_pass_on_bounds_checked_build():
    from paper_1808_10633_gb300 import build

    lib = build.build(variant="check")
    env = dict(os.environ, WB_LIBRARY=lib)
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
           os.path.join(ROOT, "tests", "test_gpu_parity.py"),
           os.path.join(ROOT, "tests", "test_gpu_linked.py"),
           os.path.join(ROOT, "tests", "test_gpu_restart.py"),
           os.path.join(ROOT, "tests", "test_gpu_learned.py"),
           "-k", "not fullsize and not gain and not training"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert "passed" in r.stdout
