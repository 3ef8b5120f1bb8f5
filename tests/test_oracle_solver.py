"""Pins of the oracle's full semi-discrete operator and integrators.

Free-stream preservation (bitwise), conservation on periodic grids,
translation / mirror / axis-permutation symmetry, the face divergence of b
under constrained transport, the exact circularly polarised Alfven wave and
the measured orders of accuracy in space and time.
"""
import numpy as np
import pytest

from paper_1808_10633_gb300 import inputs as I


def grid(orc, st, emf_mode=0):
    nx, ny, nz = st.dims
    return orc.Grid(nx, ny, nz, st.dx, st.dy, st.dz, st.gamma, emf_mode)


@pytest.mark.parametrize("emf_mode", [0, 1])
def test_free_stream_is_bitwise_steady(orc, emf_mode):
    for v, B in [((0.3, -0.2, 0.1), (0.4, -0.3, 0.2)), ((0, 0, 0), (0, 0, 0)),
                 ((1.5, 0, 0), (0, 0.7, 0))]:
        st = I.uniform(7, 6, 9, v=v, B=B)
        g = grid(orc, st, emf_mode)
        L, Lb, _ = orc.rhs(g, st.U, st.bx, st.by, st.bz)
        assert np.all(L == 0.0) and np.all(Lb == 0.0)
        U, bx, by, bz = orc.step(g, st.U, st.bx, st.by, st.bz, 1e-3)
        assert np.array_equal(U, st.U) and np.array_equal(bx, st.bx)


def test_conservation_to_roundoff(orc):
    st = I.perturbed(12, 10, 8, seed=1, jump=True)
    g = grid(orc, st)
    L, Lb, F = orc.rhs(g, st.U, st.bx, st.by, st.bz)
    for q in (0, 1, 2, 3, 7):
        scale = sum(np.abs(F[d, q]).sum() for d in range(3)) / min(st.dx, st.dy, st.dz)
        assert abs(L[q].sum()) <= 1e-14 * scale
    for d in range(3):
        assert abs(Lb[d].sum()) <= 1e-13 * np.abs(Lb[d]).sum()
    tot0 = orc.totals(g, st.U, st.bx, st.by, st.bz)
    U, bx, by, bz = orc.step(g, st.U, st.bx, st.by, st.bz, 2e-3, nsteps=3)
    tot1 = orc.totals(g, U, bx, by, bz)
    for q in range(8):
        assert abs(tot1[q] - tot0[q]) <= 1e-13 * max(1.0, np.abs(st.U[q]).mean())


def test_translation_invariance_bitwise(orc):
    st = I.perturbed(10, 9, 8, seed=2, jump=True)
    g = grid(orc, st)
    sh = (3, 2, 1)                                   # (z, y, x) shifts
    roll = lambda a: np.roll(a, sh, axis=(-3, -2, -1))
    U, bx, by, bz = orc.step(g, st.U, st.bx, st.by, st.bz, 1e-3)
    U2, bx2, by2, bz2 = orc.step(g, roll(st.U), roll(st.bx), roll(st.by), roll(st.bz), 1e-3)
    assert np.array_equal(U2, roll(U)) and np.array_equal(bx2, roll(bx))
    assert np.array_equal(by2, roll(by)) and np.array_equal(bz2, roll(bz))


def mirror(st_or_arrays, axis):
    """Mirror x_axis -> -x_axis: cells reversed, the normal momentum flips,
    B is axial so the two transverse components flip; faces normal to the
    axis move from index i to (n - i) mod n."""
    U, bx, by, bz = st_or_arrays
    ax = {0: -1, 1: -2, 2: -3}[axis]
    U = np.flip(U, axis=ax).copy()
    b = [np.flip(x, axis=ax).copy() for x in (bx, by, bz)]
    b[axis] = np.roll(b[axis], 1, axis=ax)
    U[1 + axis] *= -1
    for t in range(3):
        if t != axis:
            U[4 + t] *= -1
            b[t] *= -1
    return U, b[0], b[1], b[2]


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_mirror_symmetry(orc, axis):
    st = I.perturbed(10, 10, 10, seed=4, jump=True)
    g = grid(orc, st)
    s0 = (st.U, st.bx, st.by, st.bz)
    a = mirror(orc.step(g, *s0, 1e-3), axis)
    b = orc.step(g, *mirror(s0, axis), 1e-3)
    for x, y in zip(a, b):
        assert np.abs(x - y).max() <= 1e-13 * max(1.0, np.abs(x).max())


def test_axis_permutation_symmetry(orc):
    """(x, y, z) -> (y, z, x): the solution permutes with the axes."""
    st = I.perturbed(8, 8, 8, seed=6, jump=True)
    g = grid(orc, st)

    def perm(U, bx, by, bz):
        # new x = old y, new y = old z, new z = old x; arrays are [z, y, x]
        t = lambda a: np.transpose(a, (2, 0, 1)) if a.ndim == 3 else np.transpose(a, (0, 3, 1, 2))
        Un = t(U).copy()
        Un[[1, 2, 3]] = t(U)[[2, 3, 1]]
        Un[[4, 5, 6]] = t(U)[[5, 6, 4]]
        return Un, t(by).copy(), t(bz).copy(), t(bx).copy()

    s0 = (st.U, st.bx, st.by, st.bz)
    a = perm(*orc.step(g, *s0, 1e-3))
    b = orc.step(g, *perm(*s0), 1e-3)
    for x, y in zip(a, b):
        assert np.abs(x - y).max() <= 1e-13 * max(1.0, np.abs(x).max())


@pytest.mark.parametrize("emf_mode", [0, 1])
def test_constrained_transport_keeps_div_b(orc, emf_mode):
    st = I.turbulence(16, seed=9)
    g = grid(orc, st, emf_mode)
    d0 = orc.div_b(g, st.bx, st.by, st.bz)
    U, bx, by, bz, dts = orc.step_cfl(g, st.U, st.bx, st.by, st.bz, 0.4, nsteps=20)
    d1 = orc.div_b(g, bx, by, bz)
    bmax = max(np.abs(b).max() for b in (bx, by, bz))
    assert np.abs(d1 - d0).max() * st.dx <= 1e-14 * bmax * 20
    assert np.all(U[0] > 0)


def test_alfven_config_32cubed_exact_solution(orc):
    """Config: 32^3 unit box, amplitude 0.1, rho=1, p=0.1, B_par=1, CFL 0.4,
    10 SSP-RK3 steps; compared with the exact travelling wave."""
    st = I.alfven_wave(32, 32, 32, amp=0.1)
    g = grid(orc, st)
    U, bx, by, bz, dts = orc.step_cfl(g, st.U, st.bx, st.by, st.bz, 0.4, nsteps=10)
    t = sum(dts)
    ex = I.alfven_wave(32, 32, 32, amp=0.1, t=t)
    assert np.all(bx == 1.0)                          # normal field exactly kept
    assert np.abs(U[0] - 1.0).max() < 1e-5
    l1 = np.abs(U[5] - ex.U[5]).mean()
    assert l1 < 2e-6, l1
    # the wave is 1-D: every (y, z) column is identical
    assert np.abs(U[5] - U[5][:1, :1, :]).max() == 0.0


def _alfven_error(orc, N, T, emf_mode, amp=0.1, integrator="ssprk3", dt_scale=5.0 / 3.0, ny=1):
    st = I.alfven_wave(N, ny, ny, amp=amp)
    g = grid(orc, st, emf_mode)
    dt0 = 0.4 / (3 * 1.2 * 16)
    dt = dt0 * (16.0 / N) ** dt_scale
    n = int(np.ceil(T / dt))
    U, bx, by, bz = orc.step(g, st.U, st.bx, st.by, st.bz, T / n, nsteps=n, integrator=integrator)
    ex = I.alfven_wave(N, ny, ny, amp=amp, t=T)
    return np.abs(U[5] - ex.U[5]).mean(), U


def test_alfven_fifth_order_convergence(orc):
    """Measured order of the L1 error of B_y on the circularly polarised
    Alfven wave, dt ~ dx^(5/3) so that the third-order time error stays below
    the fifth-order space error."""
    errs = [_alfven_error(orc, N, 0.2, 0)[0] for N in (16, 32, 64)]
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders[-1] > 4.7, (errs, orders)


def test_plain_face_mean_emf_is_second_order(orc):
    """The plain four-face EMF mean loses the flux's order on grid-aligned
    waves (the reason the 1-D-consistent edge EMF is the default)."""
    errs = [_alfven_error(orc, N, 0.2, 1)[0] for N in (16, 32, 64)]
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert 1.7 < orders[-1] < 2.3, (errs, orders)


def test_thin_and_wide_transverse_extent_agree(orc):
    """ny = nz = 1 (stencil wraps onto itself) and ny = nz = 4 give the same
    1-D solution bitwise."""
    e1, U1 = _alfven_error(orc, 16, 0.05, 0, ny=1)
    e4, U4 = _alfven_error(orc, 16, 0.05, 0, ny=4)
    assert np.array_equal(U1[:, :1, :1, :], U4[:, :1, :1, :])


@pytest.mark.parametrize("integrator,order", [("ssprk3", 3.0), ("rk4", 4.0)])
def test_integrator_time_order(orc, integrator, order):
    """Fixed grid, shrinking dt: the error against a fine-dt run falls at the
    integrator's order (SSP-RK3: 3, classic RK4 of Sec. 2.1: 4)."""
    st = I.alfven_wave(16, 1, 1, amp=0.1)
    g = grid(orc, st)
    T = 0.3
    ref = orc.step(g, st.U, st.bx, st.by, st.bz, T / 1536, nsteps=1536, integrator=integrator)[0]
    errs = []
    for n in (48, 96, 192):
        U = orc.step(g, st.U, st.bx, st.by, st.bz, T / n, nsteps=n, integrator=integrator)[0]
        errs.append(np.abs(U - ref).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert abs(orders[-1] - order) < 0.35, (errs, orders)


def _scalar_weno5_upwind(f):
    """Brute-force WENO5-JS upwind interface values f_{i+1/2} of a periodic
    1-D array (candidate quadratics fitted to cell averages, exact
    smoothness integrals, paper scale x12, eps = 1e-6)."""
    from test_oracle_weno import brute_candidates

    n = len(f)
    out = np.empty(n)
    d = np.array([0.1, 0.6, 0.3])
    for i in range(n):
        st = np.array([f[(i + m) % n] for m in range(-2, 3)])
        q, IS = brute_candidates(st)
        a = d / (1e-6 + 12.0 * IS) ** 2
        out[i] = np.dot(a / a.sum(), q)
    return out


def test_entropy_wave_reduces_to_scalar_upwind_weno(orc):
    """A density (entropy) wave in uniform v, p, B is a decoupled
    characteristic field moving at u > 0.  With the local Lax-Friedrichs
    speed alpha = max |u| the '-' split flux is constant, so the mass flux is
    the scalar upwind WENO5 value of u*rho: one SSP-RK3 step of the
    oracle must equal the scalar scheme computed from first principles."""
    n = 24
    x = (np.arange(n) + 0.5) / n
    rho = 1.0 + 0.3 * np.sin(2 * np.pi * x) + 0.2 * (np.abs(x - 0.5) < 0.15)
    u = 0.7
    one = np.ones((1, 1, n))
    st = I.assemble(rho[None, None, :] * one, u * one, 0.1 * one, -0.2 * one, 0.8 * one,
                    0.5 * one, 0.3 * one, -0.4 * one, 1.0 / n, 1.0 / n, 1.0 / n)
    g = grid(orc, st)
    dt = 0.2 / n
    U1 = orc.step(g, st.U, st.bx, st.by, st.bz, dt)[0]

    def Lrho(r):
        fh = _scalar_weno5_upwind(u * r)          # flux u*rho at i+1/2
        return -(fh - np.roll(fh, 1)) * n

    r0 = rho
    r1 = r0 + dt * Lrho(r0)
    r2 = 0.75 * r0 + 0.25 * (r1 + dt * Lrho(r1))
    r3 = (1.0 / 3.0) * r0 + (2.0 / 3.0) * (r2 + dt * Lrho(r2))
    assert np.abs(U1[0, 0, 0] - r3).max() < 1e-13
    assert np.abs(U1[0, 0, 0] - r3).max() < 1e-6 * np.abs(r3 - r0).max()
