"""Two-dimensional showcase problems of Sec. 3 on the oracle (n x n x 1 grids).

Field-loop advection: a weak loop of field carried once across the periodic
unit square; the paper reports that the scheme keeps about 95 % of the
magnetic energy at t = 1 with 64 zones.  The loop problem is symmetric under
the swap x <-> y (with v = (1, 1)), which the sweeps preserve exactly.

Orszag-Tang vortex: point symmetric under (x, y) -> (1 - x, 1 - y) with
v -> -v, B -> -B; the scheme keeps that symmetry, conserves mass, momentum,
energy and the face field to round-off, and keeps the face divergence of b."""
import numpy as np

from paper_1808_10633_gb300 import inputs as I


def advance(orc, st, t_end, cfl=0.4):
    nx, ny, nz = st.dims
    g = orc.Grid(nx, ny, nz, st.dx, st.dy, st.dz, st.gamma)
    U, bx, by, bz = st.U, st.bx, st.by, st.bz
    t, steps = 0.0, 0
    while t < t_end * (1 - 1e-14):
        dt = min(orc.cfl_dt(g, U, bx, by, bz, cfl), t_end - t)
        U, bx, by, bz = orc.step(g, U, bx, by, bz, dt)
        t += dt
        steps += 1
    return g, U, bx, by, bz, steps


def magnetic_energy(U):
    return 0.5 * float((U[4] ** 2 + U[5] ** 2 + U[6] ** 2).sum())


def test_field_loop_energy_and_swap_symmetry(orc):
    st = I.field_loop(32)
    g, U, bx, by, bz, steps = advance(orc, st, 1.0)
    ratio = magnetic_energy(U) / magnetic_energy(st.U)
    # 32 zones keep less than the 95 % the paper reports at 64 zones
    assert 0.90 < ratio < 0.95, ratio
    # x <-> y swap: A_z is symmetric, so bx(j, i) = -by(i, j) (faces map onto
    # faces); rho is symmetric; both to round-off, since the two sweeps order
    # their sums differently
    assert np.abs(bx[0] + by[0].T).max() <= 1e-10 * np.abs(bx).max()
    assert np.abs(U[0, 0] - U[0, 0].T).max() <= 1e-10
    div = orc.div_b(g, bx, by, bz)
    assert np.abs(div).max() * st.dx <= 1e-14 * np.abs(st.bx).max()
    # the loop is back where it started (the error sits at the loop's edge,
    # where the field jumps, and shrinks with resolution)
    err = np.abs(bx - st.bx).sum() / np.abs(st.bx).sum()
    assert err < 0.4, err


def test_orszag_tang_symmetry_and_conservation(orc):
    st = I.orszag_tang(64)
    g, U, bx, by, bz, steps = advance(orc, st, 0.25)
    T0 = orc.totals(g, st.U, st.bx, st.by, st.bz)
    T1 = orc.totals(g, U, bx, by, bz)
    scale = orc.totals(g, np.abs(st.U), np.abs(st.bx), np.abs(st.by), np.abs(st.bz))
    assert np.all(np.abs(T1 - T0) <= 1e-13 * np.maximum(scale, 1e-3 * scale.max())), (T1 - T0, scale)
    # point symmetry: cell (i, j) <-> (n-1-i, n-1-j), vectors change sign
    flip = lambda a: a[..., ::-1, ::-1]
    for f, sgn in ((0, 1), (1, -1), (2, -1), (4, -1), (5, -1), (7, 1)):
        assert np.abs(U[f] - sgn * flip(U[f])).max() <= 1e-12 * np.abs(U[f]).max(), f
    p = (U[7] - 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0]
         - 0.5 * (U[4] ** 2 + U[5] ** 2 + U[6] ** 2)) * (st.gamma - 1)
    assert p.min() > 0 and U[0].min() > 0
    div = orc.div_b(g, bx, by, bz)
    assert np.abs(div).max() * st.dx <= 1e-13 * np.abs(st.bx).max()
