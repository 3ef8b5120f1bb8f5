"""Pins of the oracle's characteristic decomposition (Sec. 2.1, "Roe-type").

The right/left eigenvectors must diagonalise the flux Jacobian dF/dU, which
the test takes by central finite differences of the oracle's physical flux;
the flux itself is pinned by textbook special cases and, in the solver tests,
by the exact Alfven solution.  The Roe-Balsara normalisation is pinned by
its defining property: bounded, continuous eigenvectors through the
degenerate points.
"""
import numpy as np
import pytest

G = 5.0 / 3.0
SYS = [0, 1, 2, 3, 5, 6, 7]

STATES = {
    "generic": [1.2, 0.3, -0.2, 0.1, 0.7, 0.4, -0.5, 0.9],
    "negative_bn": [0.8, -0.6, 0.2, 0.4, -1.1, 0.3, 0.2, 0.5],
    "bperp_zero": [1.0, 0.1, 0.2, -0.3, 0.9, 0.0, 0.0, 0.6],
    "bn_zero": [1.3, 0.2, 0.0, 0.1, 0.0, 0.5, -0.4, 0.8],
    "hydro": [0.9, 0.4, -0.1, 0.2, 0.0, 0.0, 0.0, 1.1],
    # a^2 = gamma p / rho = bn^2 / rho  and  B_perp = 0: triple point
    "triple_point": [1.0, 0.0, 0.0, 0.0, np.sqrt(G * 0.6), 0.0, 0.0, 0.6],
    "near_triple": [1.0, 0.0, 0.0, 0.0, np.sqrt(G * 0.6), 1e-7, -2e-7, 0.6],
    "tiny_bperp": [1.0, 0.2, 0.0, 0.0, 0.5, 1e-14, 0.0, 0.3],
}


def fd_jacobian(orc, W):
    U = orc.prim_to_cons(W, G)
    A = np.zeros((7, 7))
    for c, q in enumerate(SYS):
        h = 1e-6 * max(1.0, abs(U[q]))
        Up, Um = U.copy(), U.copy()
        Up[q] += h
        Um[q] -= h
        A[:, c] = (orc.flux_n(Up, G)[SYS] - orc.flux_n(Um, G)[SYS]) / (2 * h)
    return A


@pytest.mark.parametrize("name", list(STATES))
def test_left_right_inverse(orc, name):
    lam, R, L, st = orc.eigen(np.array(STATES[name]), G)
    assert st == 0
    assert np.abs(L @ R - np.eye(7)).max() < 1e-12
    assert np.abs(R @ L - np.eye(7)).max() < 1e-12


@pytest.mark.parametrize("name", list(STATES))
def test_eigensystem_diagonalises_flux_jacobian(orc, name):
    W = np.array(STATES[name])
    lam, R, L, st = orc.eigen(W, G)
    A = fd_jacobian(orc, W)
    RAL = R @ np.diag(lam) @ L
    assert np.abs(RAL - A).max() <= 1e-7 * max(1.0, np.abs(A).max())
    assert np.all(np.diff(lam) >= -1e-14), lam      # ordered u-cf .. u+cf


def test_wave_speed_special_cases(orc):
    # field along the normal only: {cf, cs} = {a, ca}
    for rho, p, bn in [(1.0, 0.6, 0.3), (1.0, 0.1, 1.5), (2.0, 1.0, 0.9)]:
        cf, ca, cs = orc.wave_speeds([rho, 0, 0, 0, bn, 0, 0, p], G)
        a = np.sqrt(G * p / rho)
        assert ca == pytest.approx(abs(bn) / np.sqrt(rho), rel=1e-15)
        assert cf == pytest.approx(max(a, ca), rel=1e-14)
        assert cs == pytest.approx(min(a, ca), rel=1e-14)
    # no normal field: cf^2 = a^2 + |B|^2/rho, cs = 0
    cf, ca, cs = orc.wave_speeds([1.5, 0, 0, 0, 0.0, 0.3, 0.4, 0.7], G)
    assert cf == pytest.approx(np.sqrt(G * 0.7 / 1.5 + 0.25 / 1.5), rel=1e-14)
    assert ca == 0.0 and cs == 0.0


def test_hydro_flux_textbook(orc):
    rho, u, v, w, p = 1.3, 0.4, -0.2, 0.7, 0.9
    U = orc.prim_to_cons([rho, u, v, w, 0, 0, 0, p], G)
    E = p / (G - 1) + 0.5 * rho * (u * u + v * v + w * w)
    assert U[7] == pytest.approx(E, rel=1e-15)
    F = orc.flux_n(U, G)
    ref = [rho * u, rho * u * u + p, rho * u * v, rho * u * w, 0, 0, 0, (E + p) * u]
    assert np.allclose(F, ref, rtol=1e-14, atol=1e-15)


def test_induction_flux_textbook(orc):
    # F_n(B_t) = u B_t - v_t B_n, the normal flux of the normal field is zero
    W = [1.1, 0.3, -0.4, 0.2, 0.8, 0.5, -0.6, 0.7]
    F = orc.flux_n(orc.prim_to_cons(W, G), G)
    assert F[4] == 0.0
    assert F[5] == pytest.approx(0.3 * 0.5 - (-0.4) * 0.8, rel=1e-14)
    assert F[6] == pytest.approx(0.3 * (-0.6) - 0.2 * 0.8, rel=1e-14)


def _prim_R(orc, W):
    """Right eigenvectors mapped back to primitive variables (dW/dU R)."""
    lam, R, L, st = orc.eigen(np.array(W), G)
    rho, u, v, w = W[0], W[1], W[2], W[3]
    M = np.zeros((7, 7))
    M[0, 0] = 1
    M[1, 0], M[1, 1] = u, rho
    M[2, 0], M[2, 2] = v, rho
    M[3, 0], M[3, 3] = w, rho
    M[4, 4] = M[5, 5] = 1
    M[6] = [0.5 * (u * u + v * v + w * w), rho * u, rho * v, rho * w, W[5], W[6], 1 / (G - 1)]
    return np.linalg.solve(M, R)


def test_normalisation_bounded_and_continuous_at_bperp_zero(orc):
    """Roe-Balsara property: as B_perp -> 0 along a fixed direction the
    eigenvectors converge to those the degeneracy rule picks at B_perp = 0
    (direction (1,1)/sqrt2), and stay well conditioned."""
    base = [1.0, 0.1, 0.0, 0.0, 0.5, 0.0, 0.0, 0.6]     # a^2 = 1.0 > ca^2 = 0.25
    R0 = _prim_R(orc, base)
    prev = None
    for d in [1e-3, 1e-5, 1e-7]:
        W = list(base)
        W[5] = W[6] = d / np.sqrt(2)
        R = _prim_R(orc, W)
        diff = np.abs(R - R0).max()
        assert np.linalg.cond(R) < 1e3
        if prev is not None:
            assert diff < prev * 0.05
        prev = diff
    assert prev < 1e-5


def test_normalisation_continuous_through_triple_point(orc):
    """Near the triple point (B_perp -> 0 with a^2 = ca^2) the eigenvectors
    stay bounded and the decomposition stays exact."""
    for d in [1e-2, 1e-4, 1e-6, 0.0]:
        W = list(STATES["triple_point"])
        W[5] = d
        R = _prim_R(orc, W)
        assert np.isfinite(R).all()
        assert np.linalg.cond(R) < 1e4


def test_vanishing_weight_is_exactly_zero_at_bperp_zero(orc):
    """With B_perp = 0 and a^2 > ca^2 the slow weight alpha_s is exactly 0 in
    exact arithmetic; the normalisation is evaluated so that it is exactly 0
    in floating point too (not the square root of a rounding error), so the
    fast waves carry no transverse field.  With B_perp = d small, alpha_s
    grows in proportion to d (alpha_s^2 = a^2 t / ((a^2 - cs^2) D))."""
    W = np.array(STATES["bperp_zero"])               # a^2 = 1.0 > ca^2 = 0.81
    lam, R, L, st = orc.eigen(W, G)
    for f in (0, 6):                                  # fast columns; rows B_t1, B_t2
        assert R[4, f] == 0.0 and R[5, f] == 0.0
    prev = None
    for d in [1e-4, 1e-6, 1e-8]:
        Wd = W.copy()
        Wd[5] = d
        _, Rd, _, _ = orc.eigen(Wd, G)
        bt = abs(Rd[4, 0])                            # alpha_s a sqrt(rho) beta_1, beta_1 = 1
        if prev is not None:
            assert bt / prev == pytest.approx(0.01, rel=1e-6)
        prev = bt
