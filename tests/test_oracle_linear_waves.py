"""Oracle convergence on the four 1-D linear MHD waves (Sec. 3.1, Fig. 1:
fifth-order convergence of entropy, Alfven, fast and slow modes at amplitude
1e-5), with the paper's classic four-stage RK4 and dt ~ dx^(5/4) so the
fourth-order time error stays below the fifth-order space error."""
import numpy as np
import pytest

import linear_waves as LW


@pytest.mark.parametrize("mode", ["entropy", "alfven", "slow", "fast"])
def test_linear_wave_order(orc, mode):
    errs = []
    lam = LW.eigen(mode)[0]
    T = 0.25 / abs(lam)                 # a quarter period
    for N in (16, 32):
        U, bx, by, bz, dx, _ = LW.state(N, mode)
        g = orc.Grid(N, 1, 1, dx, dx, dx, LW.GAMMA, 0)
        dt0 = 0.3 * dx / (3 * 2.5)
        dt = dt0 * (N / 16.0) ** (1.0 - 5.0 / 4.0)
        n = int(np.ceil(T / dt))
        Uo = orc.step(g, U, bx, by, bz, T / n, nsteps=n, integrator="rk4")[0]
        Ue = LW.state(N, mode, t=T)[0]
        errs.append(LW.l1_error(Uo, Ue))
    order = np.log2(errs[0] / errs[1])
    assert order > 4.0, (mode, errs, order)
