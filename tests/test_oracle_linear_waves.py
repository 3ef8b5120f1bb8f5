"""Oracle convergence on the four 1-D linear MHD waves (Sec. 3.1, Fig. 1:
fifth-order convergence of entropy, Alfven, fast and slow modes at amplitude
1e-5; entropy and Alfven down to ~1e-13, where FP64 round-off stops them; the
fast and slow modes held up by wave steepening), with the paper's classic
four-stage RK4 and dt ~ dx^(5/4) so that the fourth-order time error stays
below the fifth-order space error.

Against the exact solution of the *linearised* equations, the compressive
modes stop converging at an error that does not depend on N.  That floor is
the second-order (amplitude^2) part of the nonlinear solution, i.e. the
steepening the paper names: it falls a hundredfold when the amplitude falls
tenfold, while the truncation error falls tenfold.  Measured against a finer
run of the same nonlinear problem instead (self-convergence), every mode
converges at fifth order over three refinements.  Over a full period, as in
Gardiner & Stone (2008), the second-order response of the Alfven wave is back
in its initial phase (the fast, Alfven and slow speeds of the background are
2 : 1 : 1/2), so the Alfven and entropy waves meet the linear solution to
~3e-13 at N = 128.
"""
import numpy as np
import pytest

import linear_waves as LW

pytestmark = pytest.mark.slow

NS = (16, 32, 64, 128)


@pytest.fixture(autouse=True)
def _one_thread(orc):
    """1-D grids: the oracle's row-parallel loops have one row, so one
    thread is fastest."""
    n = orc.num_threads()
    orc.set_num_threads(1)
    yield
    orc.set_num_threads(n)


def _run(orc, mode, N, amp=1e-5, periods=0.25, offset=0.5, c0=0.12):
    """RK4 run of one wave for `periods` of its period; returns the final
    state and the linear solution at the same time."""
    lam = LW.eigen(mode)[0]
    T = periods / abs(lam)
    U, bx, by, bz, dx, _ = LW.state(N, mode, amp=amp, offset=offset)
    g = orc.Grid(N, 1, 1, dx, dx, dx, LW.GAMMA, 0)
    dt = c0 * dx * (N / 16.0) ** (-0.25)
    n = int(np.ceil(T / dt))
    Uo = orc.step(g, U, bx, by, bz, T / n, nsteps=n, integrator="rk4")[0]
    return Uo, LW.state(N, mode, amp=amp, t=T, offset=offset)[0]


def _orders(errs):
    e = np.asarray(errs)
    return np.log2(e[:-1] / e[1:])


@pytest.mark.parametrize("mode", ["entropy", "alfven"])
def test_full_period_fifth_order_to_round_off(orc, mode):
    """Full period against the exact (linear) solution: fifth order over
    three refinements, below 1e-12 at N = 128 (the paper: ~1e-13)."""
    errs = [LW.l1_error(*_run(orc, mode, N, periods=1.0)) for N in NS]
    o = _orders(errs)
    assert np.all(o > 4.5), (mode, errs, o)
    assert errs[-1] < 1e-12, (mode, errs)


@pytest.mark.parametrize("mode", ["alfven", "slow", "fast"])
def test_linear_solution_floor_scales_as_amplitude_squared(orc, mode):
    """Quarter period: at N = 16 the error is truncation (linear in the
    amplitude); at N = 64 it has reached the floor, which is the amplitude^2
    part of the nonlinear solution."""
    e16 = [LW.l1_error(*_run(orc, mode, 16, amp=a)) for a in (1e-5, 1e-6)]
    e64 = [LW.l1_error(*_run(orc, mode, 64, amp=a)) for a in (1e-5, 1e-6)]
    assert 9.0 < e16[0] / e16[1] < 11.0, (mode, e16)
    assert 60.0 < e64[0] / e64[1] < 120.0, (mode, e64)


@pytest.mark.parametrize("mode", ["fast", "slow"])
def test_self_convergence_fifth_order(orc, mode):
    """Quarter period against an N = 256 run of the same nonlinear wave,
    sampled at common points (x = i/N): fifth order over three refinements,
    below 1e-12 at N = 128."""
    NR = 256
    ref = _run(orc, mode, NR, offset=0.0)[0]
    errs = [LW.l1_error(_run(orc, mode, N, offset=0.0)[0], ref[..., ::NR // N]) for N in NS]
    o = _orders(errs)
    assert np.all(o > 4.7), (mode, errs, o)
    assert errs[-1] < 1e-12, (mode, errs)
