"""The paper's claim on constrained transport (Sec. 2.1): the staggered-mesh
CT is formally second order, but with the high-order fluxes the scheme keeps
the magnetic energy density to fifth order.

* Circularly polarised Alfven wave (amplitude 0.1, rho = 1, p = 0.1,
  B_par = 1, wavelength 1): |B_perp| is constant in the exact travelling
  solution, so the magnetic energy is exactly constant; its drift after one
  period converges at fifth order with either integrator (dt ~ dx^(5/4) for
  RK4, dx^(5/3) for SSP-RK3, so the time error stays below the space error).
* Field-loop advection (Sec. 3.1, Fig. 1 right): pure advection keeps the
  energy exactly, but the field jumps at the loop's edge, so the loss
  converges at first order; 32 zones keep 93 %, 64 zones 96.5 % (the paper:
  95 % at 64 zones).
"""
import numpy as np
import pytest

from paper_1808_10633_gb300 import inputs as I

pytestmark = pytest.mark.slow


def _eb(U):
    return 0.5 * float((U[4] ** 2 + U[5] ** 2 + U[6] ** 2).sum())


@pytest.mark.parametrize("integrator,p", [("rk4", 5.0 / 4.0), ("ssprk3", 5.0 / 3.0)])
def test_alfven_magnetic_energy_fifth_order(orc, integrator, p):
    n0 = orc.num_threads()
    orc.set_num_threads(1)
    try:
        drift = []
        for N in (16, 32, 64, 128):
            st = I.alfven_wave(N, 1, 1, amp=0.1)
            g = orc.Grid(N, 1, 1, st.dx, st.dy, st.dz, st.gamma, 0)
            dt = 0.12 * st.dx * (N / 16.0) ** (1.0 - p)
            n = int(np.ceil(1.0 / dt))
            U = orc.step(g, st.U, st.bx, st.by, st.bz, 1.0 / n, nsteps=n, integrator=integrator)[0]
            drift.append(abs(_eb(U) / _eb(st.U) - 1.0))
    finally:
        orc.set_num_threads(n0)
    orders = np.log2(np.array(drift[:-1]) / np.array(drift[1:]))
    assert np.all(orders > 4.7), (drift, orders)
    assert drift[-1] < 1e-8, drift


def test_field_loop_energy_loss_first_order(orc):
    loss = []
    for n in (16, 32):
        st = I.field_loop(n)
        nx, ny, nz = st.dims
        g = orc.Grid(nx, ny, nz, st.dx, st.dy, st.dz, st.gamma)
        U, bx, by, bz = st.U, st.bx, st.by, st.bz
        t = 0.0
        while t < 1.0 * (1 - 1e-14):
            dt = min(orc.cfl_dt(g, U, bx, by, bz, 0.4), 1.0 - t)
            U, bx, by, bz = orc.step(g, U, bx, by, bz, dt)
            t += dt
        loss.append(1.0 - _eb(U) / _eb(st.U))
    assert 0.0 < loss[1] < loss[0]
    assert np.log2(loss[0] / loss[1]) > 0.8, loss
