"""Pins of the FP64 reference of the learned WENO weights (oracle/learned.py):
hand-written backprop against central finite differences, softmax and KL
properties, the detector on textbook profiles, and the linear-weight network
reproducing the fifth-order upwind flux of the printed constants."""
import os

import numpy as np
import pytest

from oracle import learned as Lr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "weno5_linear.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            k, *v = line.split()
            out[k] = [float(t) for t in v]
    return out


def _batch(n, seed):
    rng = np.random.default_rng(seed)
    x = Lr.normalise(rng.standard_normal((n, 6)))
    f5 = rng.standard_normal((n, 5))
    q = Lr.candidates(f5)
    T = q @ Lr.D_LIN + 0.05 * rng.standard_normal(n)
    return x, q, T


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = rng.standard_normal(Lr.NPARAM) * 0.3
    x, q, T = _batch(16, 2)
    L, g = Lr.loss_and_grad(p, x, q, T, 1e-2)
    idx = rng.choice(Lr.NPARAM, 60, replace=False)
    for i in idx:
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (Lr.loss_and_grad(pp, x, q, T, 1e-2)[0] - Lr.loss_and_grad(pm, x, q, T, 1e-2)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-9), i


def test_gelu_derivative_and_softmax():
    t = np.linspace(-4, 4, 81)
    fd = (Lr.gelu(t + 1e-6) - Lr.gelu(t - 1e-6)) / 2e-6
    assert np.allclose(Lr.gelu_grad(t), fd, rtol=1e-7, atol=1e-9)
    z = np.random.default_rng(3).standard_normal((50, 3)) * 5
    om = Lr.softmax(z)
    assert np.allclose(om.sum(axis=1), 1.0) and np.all(om > 0)


def test_linear_network_gives_linear_weights_and_upwind5():
    g = _golden()
    p = Lr.linear_params()
    rng = np.random.default_rng(4)
    x = Lr.normalise(rng.standard_normal((20, 6)))
    om, _ = Lr.forward(p, x)
    assert np.allclose(om, g["linear_weights"], atol=1e-15)
    cn = np.array(g["central_num"]) / g["central_den"][0]
    for _ in range(20):
        f = rng.standard_normal(5)
        D = np.diff(f)
        flux = float(np.dot(cn, f[1:5])) - Lr.phi_n_weights(*D, om[0, 0], om[0, 2])
        up5 = float(np.dot(g["upwind5_num"], f)) / g["upwind5_den"][0]
        assert flux == pytest.approx(up5, abs=1e-13)


def test_kl_term_vanishes_at_linear_weights():
    om = np.tile(Lr.D_LIN, (4, 1))
    q = np.ones((4, 3))
    assert np.allclose(Lr.record_loss(om, q, np.ones(4), 1.0), 0.0, atol=1e-15)


def test_detector_fires_on_jumps_not_on_smooth_extrema():
    h = 0.05
    xs = np.arange(-2, 3) * h
    smooth_extremum = np.diff(np.cos(xs))           # differences around a maximum
    assert not Lr.detector(smooth_extremum[None, :], 4.0)[0]
    step = np.diff(np.array([0.0, 0.0, 0.0, 1.0, 1.0]))
    assert Lr.detector(step[None, :], 4.0)[0]
    assert not Lr.detector(np.zeros((1, 4)), 4.0)[0]


def test_smoothness_gate():
    """The gate reads the Jiang-Shu smoothness indicators of Sec. 2.1.  On
    linear data all three equal 12 a^2 (no spread: the network is held back
    for any ratio above 1).  Near a critical point of the flux in general
    position they differ by O(h) relatively, on a monotone smooth stretch by
    O(h^2) (Henrick et al. 2005): the spread a ratio just above 1 tells
    apart."""
    a = 0.37
    assert Lr.smoothness_indicators([a, a, a, a]) == pytest.approx((12 * a * a,) * 3, rel=1e-15)
    assert not Lr.rough([a] * 4, 1.01)[0] and Lr.rough([a] * 4, 0.99)[0]
    spread = lambda D: max(Lr.smoothness_indicators(D)) / min(Lr.smoothness_indicators(D)) - 1.0
    # f = x^2 + x^3: a critical point at 0 with a nonzero third derivative
    # there (the O(h) term needs it); stencil off-centre by 0.3 h
    ext = [np.diff(((np.arange(-2, 3) + 0.3) * h) ** 2 + ((np.arange(-2, 3) + 0.3) * h) ** 3)
           for h in (0.04, 0.02)]
    mono = [np.diff(np.sin(0.7 + np.arange(-2, 3) * h) + 0.5 * (0.7 + np.arange(-2, 3) * h))
            for h in (0.04, 0.02)]
    assert 1.7 < spread(ext[0]) / spread(ext[1]) < 2.3             # O(h)
    assert 3.4 < spread(mono[0]) / spread(mono[1]) < 4.6           # O(h^2)
    assert Lr.rough(ext[1], 1.01)[0] and not Lr.rough(mono[1], 1.01)[0]
    assert Lr.rough(mono[1], 0.0)[0]


def test_gate_shut_gives_the_jiang_shu_flux(orc):
    """smooth above every spread: the learned reference is the oracle's
    Jiang-Shu flux (same steps, numpy instead of C)."""
    rng = np.random.default_rng(4)
    gam = 5.0 / 3.0
    P = rng.standard_normal((7, Lr.NPARAM)) * 0.5
    for t in range(5):
        W = [[1.0 + 0.1 * rng.random(), 0.2 * rng.standard_normal(), 0.2 * rng.standard_normal(),
              0.2 * rng.standard_normal(), 0.8, 0.3 * rng.standard_normal(), 0.3 * rng.standard_normal(),
              0.6 + 0.1 * rng.random()] for _ in range(6)]
        Us = np.array([orc.prim_to_cons(w, gam) for w in W])
        F = Lr.interface_flux_learned(Us, gam, P, kappa=1e30, pjump=1e30, smooth=1e300)
        Fj = orc.interface_flux(Us, gam)
        assert np.abs(F - Fj).max() <= 1e-13 * np.abs(Fj).max()


def test_learned_flux_with_linear_network_matches_upwind_on_entropy_wave(orc):
    """With omega = d and the detector off, a decoupled entropy wave's mass
    flux is the linear upwind-5 combination of u*rho."""
    g = _golden()
    gam = 5.0 / 3.0
    P = np.tile(Lr.linear_params(), (7, 1))
    rho = 1.0 + 0.2 * np.sin(np.linspace(0, 1.5, 6))
    u = 0.7
    Us = np.array([orc.prim_to_cons([r, u, 0.1, -0.2, 0.5, 0.3, -0.4, 0.8], gam) for r in rho])
    F = Lr.interface_flux_learned(Us, gam, P, kappa=1e30)
    up5 = float(np.dot(g["upwind5_num"], u * rho[:5])) / g["upwind5_den"][0]
    assert F[0] == pytest.approx(up5, rel=1e-12)
