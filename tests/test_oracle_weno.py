"""Pins of the oracle's WENO5 pieces (Sec. 2.1: phi_N, weights, eq. FWENO).

Each test checks the oracle against something other than its own formula:
the printed constants (tests/golden), the brute-force Jiang-Shu
reconstruction built from polynomial fits and exact smoothness integrals, and
the order of accuracy on smooth data.
"""
import os

import numpy as np
import pytest
from numpy.polynomial import polynomial as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "weno5_linear.txt")


def golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, *vals = line.split()
        out[key] = [float(v) for v in vals]
    return out


def brute_candidates(f):
    """Jiang-Shu candidate fluxes and smoothness integrals from first principles.

    f = f_{i-2..i+2} are treated as cell averages of h(x) on unit cells
    I_j = [j-1/2, j+1/2] (cell i at 0).  For each stencil S_k = {i-2+k .. i+k}
    fit the quadratic p_k whose cell averages are the data, evaluate it at
    x = 1/2, and integrate (p_k')^2 + (p_k'')^2 over I_i."""
    q, IS = [], []
    for k in range(3):
        cells = [-2 + k + m for m in range(3)]
        A = np.zeros((3, 3))
        for r, j in enumerate(cells):
            for n in range(3):
                # average of x^n over [j-1/2, j+1/2]
                A[r, n] = ((j + 0.5) ** (n + 1) - (j - 0.5) ** (n + 1)) / (n + 1)
        c = np.linalg.solve(A, np.array([f[j + 2] for j in cells]))
        q.append(P.polyval(0.5, c))
        d1 = P.polyder(c)
        d2 = P.polyder(c, 2)
        integ = P.polyint(P.polyadd(P.polymul(d1, d1), P.polymul(d2, d2)))
        IS.append(P.polyval(0.5, integ) - P.polyval(-0.5, integ))
    return np.array(q), np.array(IS)


def test_golden_linear_identity_brute_force():
    g = golden()
    rng = np.random.default_rng(3)
    for _ in range(20):
        f = rng.standard_normal(5)
        q, _ = brute_candidates(f)
        lin = float(np.dot(g["linear_weights"], q))
        up5 = float(np.dot(g["upwind5_num"], f)) / g["upwind5_den"][0]
        assert lin == pytest.approx(up5, abs=1e-14)


def test_linear_data_gives_linear_weights(orc):
    g = golden()
    for a in (0.0, 1e-3, 0.37, -2.5, 1e3):
        w = orc.weno_weights(a, a, a, a)
        assert np.allclose(w, g["linear_weights"], rtol=0, atol=1e-15)
        assert orc.phi_n(a, a, a, a) == 0.0


def test_phi_n_equals_brute_force_weno(orc):
    """central - phi_N(D_{i-3/2}, D_{i-1/2}, D_{i+1/2}, D_{i+3/2}) is the
    WENO5-JS upwind flux sum_k omega_k q_k, with the weights built from the
    brute-force smoothness integrals at the paper's scale (x12) and eps."""
    g = golden()
    eps = g["epsilon"][0]
    d = np.array(g["linear_weights"])
    cn = np.array(g["central_num"]) / g["central_den"][0]
    rng = np.random.default_rng(11)
    for trial in range(200):
        scale = 10.0 ** rng.uniform(-2, 2)
        f = scale * rng.standard_normal(5)
        if trial % 4 == 0:                      # a jump inside the stencil
            f[rng.integers(1, 5):] += 5 * scale
        q, IS = brute_candidates(f)
        alpha = d / (eps + 12.0 * IS) ** 2
        w = alpha / alpha.sum()
        ref = float(np.dot(w, q))
        D = np.diff(f)                          # D_{i-3/2} .. D_{i+3/2}
        central = float(np.dot(cn, f[1:5]))
        got = central - orc.phi_n(D[0], D[1], D[2], D[3])
        assert got == pytest.approx(ref, rel=1e-12, abs=1e-13 * scale)
        w0, w1, w2 = orc.weno_weights(D[0], D[1], D[2], D[3])
        assert np.allclose([w0, w1, w2], w, rtol=1e-12, atol=1e-15)


def test_minus_side_is_mirror_of_plus_side(orc):
    """The '-' term of eq. FWENO reconstructs the right-going split flux:
    on mirrored data it gives the '+' reconstruction of the mirror image."""
    g = golden()
    cn = np.array(g["central_num"]) / g["central_den"][0]
    rng = np.random.default_rng(5)
    for _ in range(50):
        f = rng.standard_normal(6)              # f_{i-2..i+3}
        D = np.diff(f)                          # D_{i-3/2} .. D_{i+5/2}
        minus = float(np.dot(cn, f[1:5])) + orc.phi_n(D[4], D[3], D[2], D[1])
        fm = f[::-1]                            # mirror about i+1/2
        Dm = np.diff(fm)
        plus_m = float(np.dot(cn, fm[1:5])) - orc.phi_n(Dm[0], Dm[1], Dm[2], Dm[3])
        assert minus == pytest.approx(plus_m, rel=1e-13, abs=1e-14)


def test_weno_flux_fifth_order_on_smooth_data(orc):
    """(Fhat_{i+1/2} - Fhat_{i-1/2}) / h approximates h'(x_i) = f'(x_i) with a
    fifth-order error on smooth data away from critical points."""
    g = golden()
    cn = np.array(g["central_num"]) / g["central_den"][0]
    x0 = 0.3
    errs = []
    hs = [0.2, 0.1, 0.05]
    for h in hs:
        def fhat(xc):                           # interface xc + h/2
            f = np.sin(xc + h * np.arange(-2, 4))
            D = np.diff(f)
            return float(np.dot(cn, f[1:5])) - orc.phi_n(D[0], D[1], D[2], D[3])
        deriv = (fhat(x0) - fhat(x0 - h)) / h
        errs.append(abs(deriv - np.cos(x0)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders.min() > 4.5, (errs, orders)


def test_weno_z_linear_data_and_brute_force_identity(orc):
    """WENO-Z keeps the linear weights on linear data, and its phi_N obeys the
    same reconstruction identity central - phi = sum_k omega_k q_k with the
    brute-force candidates."""
    g = golden()
    cn = np.array(g["central_num"]) / g["central_den"][0]
    for a in (0.0, 0.3, -2.0):
        assert np.allclose(orc.weno_weights_z(a, a, a, a), g["linear_weights"], atol=1e-15)
    rng = np.random.default_rng(21)
    for _ in range(100):
        f = rng.standard_normal(5)
        q, _ = brute_candidates(f)
        D = np.diff(f)
        w = np.array(orc.weno_weights_z(*D))
        got = float(np.dot(cn, f[1:5])) - orc.phi_n_z(*D)
        assert got == pytest.approx(float(np.dot(w, q)), rel=1e-12, abs=1e-13)


def test_critical_point_order_js_loss_and_weno_z(orc):
    """Sec. 2.1: the Jiang-Shu scheme is only third order near critical
    points; WENO-Z (the alternative it names) is not.  Max-norm error of the
    flux-difference derivative on f = sin(pi x - sin(pi x)/pi), periodic on
    [-1, 1], which has critical points with f'' != 0 (the test function of
    Henrick, Aslam & Powers 2005)."""
    g = golden()
    cn = np.array(g["central_num"]) / g["central_den"][0]

    def err(fn, N):
        x = -1 + 2 * (np.arange(N) + 0.5) / N
        h = 2.0 / N
        f = np.sin(np.pi * x - np.sin(np.pi * x) / np.pi)
        fp = np.cos(np.pi * x - np.sin(np.pi * x) / np.pi) * (np.pi - np.cos(np.pi * x))
        F = np.empty(N)
        for i in range(N):
            st = np.array([f[(i + m) % N] for m in range(-2, 3)])
            F[i] = float(np.dot(cn, st[1:5])) - fn(*np.diff(st))
        return np.abs((F - np.roll(F, 1)) / h - fp).max()

    ej = [err(orc.phi_n, N) for N in (80, 160, 320)]
    ez = [err(orc.phi_n_z, N) for N in (80, 160, 320)]
    oj = np.log2(ej[-2] / ej[-1])
    oz = np.log2(ez[-2] / ez[-1])
    assert 2.7 < oj < 3.5, (ej, oj)
    assert oz > 3.9 and ez[-1] < 0.1 * ej[-1], (ez, oz)
