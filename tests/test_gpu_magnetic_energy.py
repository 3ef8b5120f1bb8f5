"""GPU check of the paper's magnetic-energy claim (Sec. 2.1: with the
high-order fluxes the CT scheme keeps the magnetic energy density to fifth
order) and of the field-loop energy history (Sec. 3.1, Fig. 1 right), FP64.

* Circularly polarised Alfven wave, one period: the drift of the exactly
  constant magnetic energy converges at fifth order over three refinements
  (N = 16 ... 128, RK4 and SSP-RK3), and the GPU drift equals the oracle's.
* Field loop at 32^2 ... 256^2, t = 1: the energy loss falls at first order
  (the field jumps at the loop's edge); 64^2 keeps more than 95 % (the
  paper's WENO5 at 64 zones: ~95 %).
"""
import numpy as np
import pytest

from paper_1808_10633_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wb():
    from paper_1808_10633_gb300 import build, wombat

    build.build()
    return wombat


def _eb(U):
    return 0.5 * float((U[4] ** 2 + U[5] ** 2 + U[6] ** 2).sum())


def _alfven(wb, N, integrator, p):
    st = I.alfven_wave(N, 1, 1, amp=0.1)
    g = wb.Grid.from_state(st, precision="fp64", integrator=integrator)
    dt = 0.04 * st.dx * (N / 16.0) ** (1.0 - p)
    n = int(np.ceil(1.0 / dt))
    g.step(1.0 / n, n)
    U = g.get_state_single()[0]
    g.close()
    return st, U, 1.0 / n, n


@pytest.mark.parametrize("integrator,p", [("rk4", 5.0 / 4.0), ("ssprk3", 5.0 / 3.0)])
def test_gpu_alfven_magnetic_energy_fifth_order(wb, integrator, p):
    drift = []
    for N in (16, 32, 64, 128):
        st, U, _, _ = _alfven(wb, N, integrator, p)
        drift.append(abs(_eb(U) / _eb(st.U) - 1.0))
    orders = np.log2(np.array(drift[:-1]) / np.array(drift[1:]))
    assert np.all(orders > 4.7), (drift, orders)
    assert drift[-1] < 1e-8, drift


def test_gpu_alfven_magnetic_energy_matches_oracle(orc, wb):
    st, U, dt, n = _alfven(wb, 32, "rk4", 5.0 / 4.0)
    g = orc.Grid(32, 1, 1, st.dx, st.dy, st.dz, st.gamma, 0)
    Uo = orc.step(g, st.U, st.bx, st.by, st.bz, dt, nsteps=n, integrator="rk4")[0]
    d_gpu = _eb(U) / _eb(st.U) - 1.0
    d_orc = _eb(Uo) / _eb(st.U) - 1.0
    assert abs(d_gpu - d_orc) <= 1e-6 * abs(d_orc), (d_gpu, d_orc)


def test_gpu_field_loop_energy_loss(wb):
    loss = []
    for n in (32, 64, 128, 256):
        st = I.field_loop(n)
        g = wb.Grid.from_state(st, precision="fp64")
        t = 0.0
        while t < 1.0 * (1 - 1e-14):
            dt = min(g.cfl_dt(0.4), 1.0 - t)
            g.step(dt, 1)
            t += dt
        U = g.get_state_single()[0]
        g.close()
        loss.append(1.0 - _eb(U) / _eb(st.U))
    orders = np.log2(np.array(loss[:-1]) / np.array(loss[1:]))
    assert np.all(np.diff(loss) < 0) and loss[-1] > 0, loss
    assert np.all(orders > 0.7), (loss, orders)
    assert loss[1] < 0.05, loss
