"""GPU convergence on the four 1-D linear MHD waves (Sec. 3.1, Fig. 1),
FP64 path with the paper's classic RK4, dt ~ dx^(5/4), a quarter period.
The entropy wave converges at fifth order to round-off level; the other
three converge at fifth order until the second-order (amplitude^2, 1e-10)
terms of the nonlinear equations dominate, as the paper reports for the
compressive modes.  The GPU errors match the oracle's at N = 32."""
import numpy as np
import pytest

import linear_waves as LW

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wb():
    from paper_1808_10633_gb300 import build, wombat

    build.build()
    return wombat


def _run(wb, mode, N):
    lam = LW.eigen(mode)[0]
    T = 0.25 / abs(lam)
    U, bx, by, bz, dx, _ = LW.state(N, mode)
    g = wb.Grid([(N, 1, 1)], dx, dx, dx, U, np.stack([bx, by, bz]), gamma=LW.GAMMA,
                precision="fp64", integrator="rk4")
    dt = 0.3 * dx / (3 * 2.5) * (N / 16.0) ** (1.0 - 5.0 / 4.0)
    n = int(np.ceil(T / dt))
    g.step(T / n, n)
    Ug = g.get_state_single()[0]
    g.close()
    return Ug, LW.l1_error(Ug, LW.state(N, mode, t=T)[0]), T / n, n


@pytest.mark.parametrize("mode", ["entropy", "alfven", "slow", "fast"])
def test_gpu_linear_wave_convergence(wb, mode):
    errs = [_run(wb, mode, N)[1] for N in (16, 32, 64, 128)]
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders[0] > 4.0, (errs, orders)
    if mode == "entropy":
        assert orders[1] > 4.5 and errs[2] < 1e-11, (errs, orders)
    else:
        assert errs[2] < 2e-10, errs


def test_gpu_linear_wave_matches_oracle(orc, wb):
    for mode in ("alfven", "fast"):
        Ug, eg, dt, n = _run(wb, mode, 32)
        U, bx, by, bz, dx, _ = LW.state(32, mode)
        g = orc.Grid(32, 1, 1, dx, dx, dx, LW.GAMMA, 0)
        Uo = orc.step(g, U, bx, by, bz, dt, nsteps=n, integrator="rk4")[0]
        eo = LW.l1_error(Uo, LW.state(32, mode, t=dt * n)[0])
        assert abs(eg - eo) <= 1e-3 * eo, (mode, eg, eo)
        assert np.abs(Ug - Uo).max() <= 1e-13
