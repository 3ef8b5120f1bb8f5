"""The operation-counting build of the oracle (oracle/count_ops.cpp).

It compiles the oracle's own source with a counting value type for double,
so its results must be bit-identical to the plain oracle's; its counts are
pinned by a hand count of the printed interpolant (Sec. 2.1) and give the
algorithmic operation counts per interface and per zone update that the
design notes quote."""
import numpy as np
import pytest

import oracle as O
from oracle import counts as C
from paper_1808_10633_gb300 import inputs as I


def test_phi_n_count_matches_hand_count_of_the_formula():
    """phi_N with the Jiang-Shu weights, read off Sec. 2.1 as written in the
    oracle: IS_0 5 add 6 mul, IS_1 5 add 4 mul, IS_2 5 add 6 mul, the three
    alpha_k 6 add 3 mul 3 div, their sum 2 add, omega_0..2 3 div, the
    interpolant 6 add 4 mul 2 div: 29 add, 23 mul, 8 div."""
    for args in [(0.3, -0.2, 0.7, 0.11), (1.5, 2.25, -3.0, 0.375)]:
        v, n = C.phi_n(*args)
        assert v == O.phi_n(*args)
        assert n == {"add": 29, "mul": 23, "div": 8, "sqrt": 0}
    # structural zeros are free: all-zero differences leave only the eps
    # terms, the reciprocals and the weight divisions
    _, n0 = C.phi_n(0.0, 0.0, 0.0, 0.0)
    assert n0["add"] < 29 and n0["mul"] < 23 and n0["div"] == 8


def _turb(n=16, seed=3):
    st = I.turbulence(n, seed=seed)
    g = O.Grid(n, n, n, st.dx, st.dy, st.dz)
    return st, g


def test_counted_interface_flux_is_the_oracle_and_costs_3931_flops():
    st, g = _turb()
    U = O.cell_b(g, st.U, st.bx, st.by, st.bz)
    Us = np.stack([U[:, 2, 3, (5 + m - 3) % 16] for m in range(6)])   # x stencil: global = normal frame
    F, n = C.interface_flux(Us)
    assert np.array_equal(F, O.interface_flux(Us))
    assert n == {"add": 1756, "mul": 1941, "div": 200, "sqrt": 34}
    assert C.flops(n) == 3931
    W = 0.5 * (O.cons_to_prim(Us[2]) + O.cons_to_prim(Us[3]))
    (_, _, _, status), ne = C.eigen(W)
    assert status == 0
    # eigen-structure incl. the numerical inverse of R (the oracle's L)
    assert C.flops(ne) == 885


def test_counted_step_is_the_oracle_and_costs_36420_flops_per_zone():
    st, g = _turb()
    gc = g.c()
    U, bx, by, bz = [a.copy() for a in (st.U, st.bx, st.by, st.bz)]
    dt = 1e-3
    n = C.ssprk3_step(gc, dt, U, bx, by, bz)
    ref = O.step(g, st.U, st.bx, st.by, st.bz, dt)
    for a, b in zip((U, bx, by, bz), ref):
        assert np.array_equal(a, b)
    per_zone = C.flops(n) / 16 ** 3
    assert per_zone == pytest.approx(36420.33, abs=0.01)
