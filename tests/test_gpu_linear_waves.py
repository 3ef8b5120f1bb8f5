"""GPU convergence on the four 1-D linear MHD waves (Sec. 3.1, Fig. 1), FP64
path with the paper's classic RK4 and dt ~ dx^(5/4), run for a full period
as Gardiner & Stone (2008) do, amplitude 1e-5.

* Entropy and Alfven waves against the exact (linear) solution: fifth order
  over three refinements, down to ~1e-13 at N = 128-256 where FP64 round-off
  stops them (the paper's figure).
* Fast and slow waves: against the linear solution they stop at an N-
  independent floor, the amplitude^2 (steepening) part of the nonlinear
  solution, which falls a hundredfold for a tenfold smaller amplitude;
  against an N = 256 run of the same nonlinear problem they converge at
  fifth order over three refinements, to ~1e-11 at N = 64 (the paper:
  WENO5 reaches 1e-11 at 64 zones) and below 1e-12 at N = 128.
* The GPU errors match the oracle's at N = 32.
"""
import numpy as np
import pytest

import linear_waves as LW

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wb():
    from paper_1808_10633_gb300 import build, wombat

    build.build()
    return wombat


def _run(wb, mode, N, amp=1e-5, periods=1.0, offset=0.5):
    """(final state, linear solution at the same time, dt, steps)."""
    lam = LW.eigen(mode)[0]
    T = periods / abs(lam)
    U, bx, by, bz, dx, _ = LW.state(N, mode, amp=amp, offset=offset)
    g = wb.Grid([(N, 1, 1)], dx, dx, dx, U, np.stack([bx, by, bz]), gamma=LW.GAMMA,
                precision="fp64", integrator="rk4")
    dt = 0.3 * dx / (3 * 2.5) * (N / 16.0) ** (1.0 - 5.0 / 4.0)
    n = int(np.ceil(T / dt))
    g.step(T / n, n)
    Ug = g.get_state_single()[0]
    g.close()
    return Ug, LW.state(N, mode, amp=amp, t=T, offset=offset)[0], T / n, n


def _orders(errs):
    e = np.asarray(errs)
    return np.log2(e[:-1] / e[1:])


@pytest.mark.parametrize("mode", ["entropy", "alfven"])
def test_gpu_full_period_fifth_order_to_round_off(wb, mode):
    errs = [LW.l1_error(*_run(wb, mode, N)[:2]) for N in (16, 32, 64, 128, 256)]
    o = _orders(errs)
    assert np.all(o[:3] > 4.5), (mode, errs, o)
    assert errs[3] < 1e-12 and errs[4] < 1e-12, (mode, errs)


@pytest.mark.parametrize("mode", ["fast", "slow"])
def test_gpu_self_convergence_fifth_order(wb, mode):
    NR = 256
    ref = _run(wb, mode, NR, offset=0.0)[0]
    errs = [LW.l1_error(_run(wb, mode, N, offset=0.0)[0], ref[..., ::NR // N]) for N in (16, 32, 64, 128)]
    o = _orders(errs)
    assert np.all(o > 4.5), (mode, errs, o)
    # the paper: WENO5 reaches L1 errors of 1e-11 at 64 zones
    assert errs[2] < 1.5e-11 and errs[3] < 1e-12, (mode, errs)


@pytest.mark.parametrize("mode", ["fast", "slow"])
def test_gpu_linear_solution_floor_scales_as_amplitude_squared(wb, mode):
    e = [LW.l1_error(*_run(wb, mode, 128, amp=a)[:2]) for a in (1e-5, 1e-6)]
    assert 60.0 < e[0] / e[1] < 120.0, (mode, e)


def test_gpu_linear_wave_matches_oracle(orc, wb):
    for mode in ("alfven", "fast"):
        Ug, Ue, dt, n = _run(wb, mode, 32, periods=0.25)
        eg = LW.l1_error(Ug, Ue)
        U, bx, by, bz, dx, _ = LW.state(32, mode)
        g = orc.Grid(32, 1, 1, dx, dx, dx, LW.GAMMA, 0)
        Uo = orc.step(g, U, bx, by, bz, dt, nsteps=n, integrator="rk4")[0]
        eo = LW.l1_error(Uo, LW.state(32, mode, t=dt * n)[0])
        assert abs(eg - eo) <= 1e-3 * eo, (mode, eg, eo)
        assert np.abs(Ug - Uo).max() <= 1e-13
