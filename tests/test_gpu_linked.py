"""Linked brick patches on the GPU: a world cut into uneven bricks that read
their neighbours' cells in place advances exactly as the uncut world.

Each interface's flux, each edge EMF and each cell update sees the same
input values in the same order whether its cells sit in one patch or in
several, so the results are compared bit for bit with the single-grid run;
the single grid itself is held to the oracle."""
import numpy as np
import pytest

from paper_1808_10633_gb300 import bricks, inputs as I

pytestmark = pytest.mark.gpu

CUTS = ([0, 11, 25, 40], [0, 17, 36], [0, 9, 28])


@pytest.fixture(scope="module")
def wb():
    from paper_1808_10633_gb300 import build, wombat

    build.build()
    return wombat


@pytest.fixture(scope="module")
def world():
    return I.perturbed(40, 36, 28, seed=91, jump=True)


def run(wb, st, cuts, nsteps, dt, **kw):
    if cuts is None:
        g = wb.Grid.from_state(st, **kw)
    else:
        g = wb.Grid.from_bricks(st, cuts, **kw)
    g.step(dt, nsteps)
    U, b = g.get_state()
    T = g.totals()
    g.close()
    if cuts is not None:
        U, b = bricks.join(U, b, cuts)
    return U.reshape((8,) + st.shape), b.reshape((3,) + st.shape), T


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_bricks_match_single_grid_bitwise(wb, world, precision):
    U1, b1, T1 = run(wb, world, None, 3, 2e-3, precision=precision)
    U2, b2, T2 = run(wb, world, CUTS, 3, 2e-3, precision=precision)
    assert np.array_equal(U1, U2) and np.array_equal(b1, b2)
    assert np.allclose(T1, T2, rtol=1e-13, atol=1e-15 * np.abs(T1).max())


def test_bricks_match_oracle(orc, wb, world):
    U2, b2, _ = run(wb, world, CUTS, 2, 2e-3, precision="fp64")
    nx, ny, nz = world.dims
    og = orc.Grid(nx, ny, nz, world.dx, world.dy, world.dz, world.gamma)
    Uo, bxo, byo, bzo = orc.step(og, world.U, world.bx, world.by, world.bz, 2e-3, nsteps=2)
    floor = 1e-3 * np.abs(Uo).max()
    for f in range(8):
        assert np.abs(U2[f] - Uo[f]).max() <= 1e-12 * max(np.abs(Uo[f]).max(), floor), f
    bo = np.stack([bxo, byo, bzo])
    assert np.abs(b2 - bo).max() <= 1e-12 * np.abs(bo).max()


def test_bricks_rk4_mean_emf_cfl_and_autotune(wb, world):
    kw = dict(precision="fp64", integrator="rk4", emf_mode=1)
    g1 = wb.Grid.from_state(world, **kw)
    g2 = wb.Grid.from_bricks(world, CUTS, **kw)
    assert g1.cfl_dt(0.4) == g2.cfl_dt(0.4)
    ms = g2.autotune()
    assert ms.shape == (3, 5)
    for g in (g1, g2):
        g.step_cfl(0.4, 3)
    U1, b1 = g1.get_state()
    U2, b2 = bricks.join(*g2.get_state(), CUTS)
    g1.close()
    g2.close()
    assert np.array_equal(U1.reshape(U2.shape), U2) and np.array_equal(b1.reshape(b2.shape), b2)


def test_bricks_2d_thin_axis_and_weno_z(wb):
    st = I.orszag_tang(48)
    cuts = ([0, 13, 30, 48], [0, 20, 48], [0, 1])
    for weights in ("js", "z"):
        U1, b1, _ = run(wb, st, None, 5, 1e-3, precision="fp64", weights=weights)
        U2, b2, _ = run(wb, st, cuts, 5, 1e-3, precision="fp64", weights=weights)
        assert np.array_equal(U1, U2) and np.array_equal(b1, b2), weights


def test_bricks_learned_weights(wb, world):
    from paper_1808_10633_gb300 import learned as Ln

    params = Ln.init_params(seed=3)
    params = (params + 0.3 * np.random.default_rng(4).standard_normal(params.shape)).astype(np.float32)
    out = []
    for cuts in (None, CUTS):
        g = wb.Grid.from_state(world, precision="learned") if cuts is None else \
            wb.Grid.from_bricks(world, cuts, precision="learned")
        g.set_mlp(params, 4.0, 0.5)
        g.step(2e-3, 2)
        U, b = g.get_state()
        g.close()
        if cuts is not None:
            U, b = bricks.join(U, b, cuts)
        out.append((U.reshape(-1), b.reshape(-1)))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
