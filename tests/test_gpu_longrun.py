"""Many steps: 400 CFL steps (about one sound crossing) of the 48^3 decaying
turbulence in FP64 and FP32.  The scheme is conservative and the
constrained transport keeps the face divergence of b at round-off, so over
the whole run: mass, momentum and energy totals move only by round-off
(FP64: 1e-12 of their scale; FP32: 2e-5), max |div b| stays at round-off of
max |b| / dx, the state stays finite with rho, p > 0 (the CFL reduction
checks every step's start state), and FP32 tracks FP64 in the L1 norm of
each field to 1e-3 relative (turbulence amplifies round-off differences, so
the bound is looser than after 20 steps)."""
import numpy as np
import pytest

from paper_1808_10633_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wb():
    from paper_1808_10633_gb300 import build, wombat

    build.build()
    return wombat


@pytest.fixture(scope="module")
def runs(wb):
    st = I.turbulence(48, seed=77)
    out = {}
    for prec in ("fp64", "fp32"):
        g = wb.Grid.from_state(st, precision=prec)
        t0 = g.totals()
        g.step_cfl(0.4, 400)
        t1 = g.totals()
        div, bmax = g.div_b()
        U = g.get_state()[0].reshape(8, -1)
        info = g.info()
        g.close()
        out[prec] = (t0, t1, div, bmax, U, info)
    return st, out


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_totals_and_div_b_hold_over_400_steps(runs, prec, tol):
    st, out = runs
    t0, t1, div, bmax, U, info = out[prec]
    assert info["steps"] == 400 and info["time"] > 0.3
    assert np.all(np.isfinite(U)) and U[0].min() > 0
    scale = np.maximum(np.abs(t0), 1e-3 * np.abs(t0).max())
    rel = np.abs(t1 - t0) / scale
    # rho, momentum, energy and the face sums of b are conserved
    assert rel.max() <= tol, rel
    assert div <= (1e-12 if prec == "fp64" else 2e-5) * bmax / st.dx, (div, bmax)


def test_fp32_tracks_fp64_over_400_steps(runs):
    st, out = runs
    U64, U32 = out["fp64"][4], out["fp32"][4]
    for f in range(8):
        l1 = np.abs(U32[f] - U64[f]).mean() / max(np.abs(U64[f]).mean(), 1e-30)
        assert l1 <= 1e-3, (f, l1)
