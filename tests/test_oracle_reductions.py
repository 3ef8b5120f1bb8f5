"""Pins of the CFL time step and the conserved totals: brute force in exact
rational or 50-digit arithmetic on tiny grids."""
from fractions import Fraction

import numpy as np
import pytest

from paper_1808_10633_gb300 import inputs as I

mpmath = pytest.importorskip("mpmath")


def test_cfl_dt_brute_force(orc):
    mpmath.mp.dps = 50
    st = I.perturbed(3, 4, 5, seed=12, jump=True)
    nx, ny, nz = st.dims
    g = orc.Grid(nx, ny, nz, st.dx, st.dy, st.dz, st.gamma)
    U = orc.cell_b(g, st.U, st.bx, st.by, st.bz)
    gam = mpmath.mpf(5) / 3
    smax = mpmath.mpf(0)
    dxs = [mpmath.mpf(st.dx), mpmath.mpf(st.dy), mpmath.mpf(st.dz)]
    for c in np.ndindex(st.shape):
        q = [mpmath.mpf(float(U[f][c])) for f in range(8)]
        rho = q[0]
        v = [q[1] / rho, q[2] / rho, q[3] / rho]
        B = q[4:7]
        p = (gam - 1) * (q[7] - (q[1] * v[0] + q[2] * v[1] + q[3] * v[2]) / 2
                         - (B[0] ** 2 + B[1] ** 2 + B[2] ** 2) / 2)
        a2 = gam * p / rho
        b2 = (B[0] ** 2 + B[1] ** 2 + B[2] ** 2) / rho
        s = mpmath.mpf(0)
        for d in range(3):
            ca2 = B[d] ** 2 / rho
            cf = mpmath.sqrt((a2 + b2 + mpmath.sqrt((a2 + b2) ** 2 - 4 * a2 * ca2)) / 2)
            s += (abs(v[d]) + cf) / dxs[d]
        smax = max(smax, s)
    ref = float(mpmath.mpf("0.4") / smax)
    got = orc.cfl_dt(g, st.U, st.bx, st.by, st.bz, 0.4)
    assert got == pytest.approx(ref, rel=4e-15)


def test_totals_exact_rational(orc):
    st = I.perturbed(4, 3, 5, seed=13)
    nx, ny, nz = st.dims
    g = orc.Grid(nx, ny, nz, st.dx, st.dy, st.dz, st.gamma)
    U = orc.cell_b(g, st.U, st.bx, st.by, st.bz)
    got = orc.totals(g, st.U, st.bx, st.by, st.bz)
    dV = Fraction(st.dx) * Fraction(st.dy) * Fraction(st.dz)
    for q in range(8):
        exact = sum((Fraction(float(x)) for x in U[q].ravel()), Fraction(0)) * dV
        assert got[q] == pytest.approx(float(exact), rel=2e-16, abs=1e-300)


def test_cell_b_is_face_mean(orc):
    st = I.perturbed(5, 4, 3, seed=14)
    nx, ny, nz = st.dims
    g = orc.Grid(nx, ny, nz, st.dx, st.dy, st.dz, st.gamma)
    U = orc.cell_b(g, st.U, st.bx, st.by, st.bz)
    assert np.array_equal(U[4], 0.5 * (st.bx + np.roll(st.bx, -1, axis=2)))
    assert np.array_equal(U[5], 0.5 * (st.by + np.roll(st.by, -1, axis=1)))
    assert np.array_equal(U[6], 0.5 * (st.bz + np.roll(st.bz, -1, axis=0)))


def test_totals_recover_the_digits_a_plain_sum_loses(orc):
    """Sum 1e16 + 1 - 1e16 + 1 (and shuffled sign patterns) along the cells:
    the exact total is 2 (and so on), which a plain left-to-right FP64 sum
    misses (1e16 + 1 rounds to 1e16).  The compensated sum is exact here, and
    the same bits on every IEEE host."""
    g = orc.Grid(4, 1, 1, 1.0, 1.0, 1.0)
    U = np.zeros((8, 1, 1, 4))
    U[0] = 1.0
    bz = np.zeros((1, 1, 4))
    for vals, exact in (([1e16, 1.0, -1e16, 1.0], 2.0), ([1.0, 1e16, 1.0, -1e16], 2.0),
                        ([3.0, 2.0 ** 60, -(2.0 ** 60), 0.5], 3.5)):
        U[0, 0, 0] = vals
        got = orc.totals(g, U, bz, bz, bz)
        assert got[0] == exact, (vals, got[0])
    # a plain sum of the first pattern would give 1
    assert ((1e16 + 1.0) - 1e16) + 1.0 == 1.0
