"""GPU path vs the FP64 CPU oracle, through the C ABI.

Tolerances: FP64 must match the oracle to 1e-12 relative per step, with the
relative error of a field taken as max|GPU - oracle| / max|oracle field|;
a field that vanishes in exact arithmetic (e.g. m_x of the Alfven wave, made
of round-off only) is measured against a floor of 1e-3 of the largest field
of the state instead of its own noise.  The GPU sums
differently ordered but algebraically identical expressions, so the
expected mismatch is a few ulps times the condition of the WENO weights.
FP32 runs are compared per field by L1 relative to the FP64 oracle."""
import numpy as np
import pytest

from paper_1808_10633_gb300 import inputs as I
from sampling import oracle_face_flux

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def wb():
    from paper_1808_10633_gb300 import build, wombat

    build.build()
    return wombat


def ogrid(orc, st, emf_mode=0):
    nx, ny, nz = st.dims
    return orc.Grid(nx, ny, nz, st.dx, st.dy, st.dz, st.gamma, emf_mode)


def rel_err(gpu, ref):
    out = []
    floor = 1e-3 * max(np.abs(ref).max(), 1e-300)
    for f in range(gpu.shape[0]):
        scale = max(np.abs(ref[f]).max(), floor)
        out.append(np.abs(gpu[f] - ref[f]).max() / scale)
    return np.array(out)


def compare(orc, wb, st, dt, nsteps=1, emf_mode=0, integrator="ssprk3", tol=TOL64):
    g = wb.Grid.from_state(st, precision="fp64", emf_mode=emf_mode, integrator=integrator)
    g.step(dt, nsteps)
    U, bx, by, bz = g.get_state_single()
    g.close()
    Uo, bxo, byo, bzo = orc.step(ogrid(orc, st, emf_mode), st.U, st.bx, st.by, st.bz, dt,
                                 nsteps=nsteps, integrator=integrator)
    eU = rel_err(U, Uo)
    eb = rel_err(np.stack([bx, by, bz]), np.stack([bxo, byo, bzo]))
    assert eU.max() <= tol and eb.max() <= tol, (eU, eb)
    return eU, eb


@pytest.mark.parametrize("dims", [(40, 20, 12), (16, 16, 16), (33, 9, 17), (7, 37, 5)])
def test_fp64_one_step_ragged_tiles(orc, wb, dims):
    st = I.perturbed(*dims, seed=sum(dims), jump=True)
    compare(orc, wb, st, 2e-3)


def test_fp64_large_magnitude_state(orc, wb):
    """Ideal MHD is unchanged by v, B -> V v, V B, p, E -> V^2 p, V^2 E and
    t -> t / V.  At V = 1e9 the energy fluxes reach ~1e27, the smoothness
    indicators ~1e54 and the product of the two weight denominators of a
    field's phi_N pair overflows FP64, so the FP64 sweep takes its path with
    one division per side; the step must still match the oracle."""
    V = 1e9
    st = I.perturbed(24, 12, 10, seed=31, jump=True)
    U = st.U.copy()
    U[1:7] *= V
    U[7] *= V * V
    big = I.State(U, st.bx * V, st.by * V, st.bz * V, st.dx, st.dy, st.dz, st.gamma, st.meta)
    compare(orc, wb, big, 2e-3 / V)


def test_fp64_three_steps_emf_modes(orc, wb):
    st = I.perturbed(24, 20, 16, seed=5, jump=True)
    compare(orc, wb, st, 2e-3, nsteps=3, emf_mode=0)
    compare(orc, wb, st, 2e-3, nsteps=3, emf_mode=1)


def test_fp64_rk4(orc, wb):
    st = I.perturbed(20, 16, 12, seed=8, jump=True)
    compare(orc, wb, st, 2e-3, nsteps=2, integrator="rk4")


def test_fp64_turbulence_cfl_steps(orc, wb):
    st = I.turbulence(32, seed=1808)
    g = wb.Grid.from_state(st, precision="fp64")
    g.step_cfl(0.4, 4)
    U, bx, by, bz = g.get_state_single()
    t_gpu = g.info()["time"]
    g.close()
    Uo, bxo, byo, bzo, dts = orc.step_cfl(ogrid(orc, st), st.U, st.bx, st.by, st.bz, 0.4, nsteps=4)
    assert t_gpu == pytest.approx(sum(dts), rel=1e-13)
    eU = rel_err(U, Uo)
    eb = rel_err(np.stack([bx, by, bz]), np.stack([bxo, byo, bzo]))
    assert eU.max() <= TOL64 and eb.max() <= TOL64, (eU, eb)


def test_alfven_config_fp64(orc, wb):
    """32^3 Alfven wave, CFL 0.4, 10 steps: parity with the oracle and the
    exact solution."""
    st = I.alfven_wave(32, 32, 32, amp=0.1)
    g = wb.Grid.from_state(st, precision="fp64")
    g.step_cfl(0.4, 10)
    U, bx, by, bz = g.get_state_single()
    t = g.info()["time"]
    g.close()
    Uo, bxo, byo, bzo, dts = orc.step_cfl(ogrid(orc, st), st.U, st.bx, st.by, st.bz, 0.4, nsteps=10)
    assert rel_err(U, Uo).max() <= TOL64
    assert np.all(bx == 1.0)
    ex = I.alfven_wave(32, 32, 32, amp=0.1, t=t)
    assert np.abs(U[5] - ex.U[5]).mean() < 2e-6


def test_cfl_dt_and_totals(orc, wb):
    st = I.turbulence(24, seed=3)
    g = wb.Grid.from_state(st, precision="fp64")
    dt = g.cfl_dt(0.4)
    tot = g.totals()
    g.close()
    og = ogrid(orc, st)
    assert dt == pytest.approx(orc.cfl_dt(og, st.U, st.bx, st.by, st.bz, 0.4), rel=1e-14)
    ref = orc.totals(og, st.U, st.bx, st.by, st.bz)
    scale = np.abs(st.U).reshape(8, -1).sum(axis=1) * st.dx * st.dy * st.dz
    assert np.all(np.abs(tot - ref) <= 1e-14 * np.maximum(scale, 1e-300)), (tot, ref)


def test_totals_deterministic_and_conserved(wb):
    st = I.turbulence(32, seed=4)
    g = wb.Grid.from_state(st, precision="fp64")
    t0 = g.totals()
    assert np.array_equal(t0, g.totals())
    g.step_cfl(0.4, 3)
    t1 = g.totals()
    g.close()
    scale = np.abs(st.U).reshape(8, -1).sum(axis=1) * st.dx * st.dy * st.dz
    assert np.all(np.abs(t1 - t0) <= 1e-13 * scale), (t1 - t0)


def test_batched_patches_fp64(orc, wb):
    sts = I.patch_batch(5, seed=2, lo=8, hi=20)
    g = wb.Grid.from_patches(sts, precision="fp64")
    dt = 0.2 * min(orc.cfl_dt(ogrid(orc, s), s.U, s.bx, s.by, s.bz, 1.0) for s in sts)
    g.step(dt, 2)
    U, b = g.get_state()
    g.close()
    oU = ob = 0
    for s in sts:
        n = s.U[0].size
        Uo, bxo, byo, bzo = orc.step(ogrid(orc, s), s.U, s.bx, s.by, s.bz, dt, nsteps=2)
        Ug = U[oU:oU + 8 * n].reshape(Uo.shape)
        bg = b[ob:ob + 3 * n].reshape((3,) + s.shape)
        oU += 8 * n
        ob += 3 * n
        assert rel_err(Ug, Uo).max() <= TOL64
        assert rel_err(bg, np.stack([bxo, byo, bzo])).max() <= TOL64


def test_thin_grid_and_free_stream(orc, wb):
    st = I.alfven_wave(16, 1, 1, amp=0.1)
    compare(orc, wb, st, 2e-3, nsteps=2)
    st = I.uniform(9, 5, 3)
    g = wb.Grid.from_state(st, precision="fp64")
    g.step(1e-2, 3)
    U, bx, by, bz = g.get_state_single()
    g.close()
    assert np.abs(U - st.U).max() <= 4e-16 * np.abs(st.U).max()
    assert np.array_equal(bx, st.bx) or np.abs(bx - st.bx).max() <= 4e-16


def test_fp32_close_to_fp64_oracle(orc, wb):
    st = I.turbulence(32, seed=11)
    g = wb.Grid.from_state(st, precision="fp32")
    dt = orc.cfl_dt(ogrid(orc, st), st.U, st.bx, st.by, st.bz, 0.4)
    g.step(dt, 3)
    U, bx, by, bz = g.get_state_single()
    g.close()
    Uo, bxo, byo, bzo = orc.step(ogrid(orc, st), st.U, st.bx, st.by, st.bz, dt, nsteps=3)
    for f in range(8):
        l1 = np.abs(U[f] - Uo[f]).mean() / max(np.abs(Uo[f]).mean(), 1e-30)
        assert l1 < 1e-5, (f, l1)


def test_nonfinite_state_is_reported(wb):
    st = I.perturbed(8, 8, 8, seed=1)
    st.U[0, 3, 3, 3] = np.nan
    g = wb.Grid.from_state(st, precision="fp64")
    with pytest.raises(wb.WombatError) as e:
        g.cfl_dt(0.4)
    assert e.value.code == wb.WB_ENONFINITE
    g.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-4)])
def test_fullsize_256_sampled_interfaces(orc, wb, prec, tol):
    """At the benchmark's 256^3 turbulence size, in the benchmark's launch
    configuration, 200 random interfaces per axis agree with the oracle's
    single-interface flux."""
    st = I.turbulence(256, seed=1808)
    g = wb.Grid.from_state(st, precision=prec)
    rng = np.random.default_rng(99)
    nx, ny, nz = st.dims
    for axis in range(3):
        F = g.face_fluxes(axis)
        idx = rng.integers(0, [nx, ny, nz], size=(200, 3))
        got = np.empty((200, 7))
        ref = np.empty((200, 7))
        for r, (i, j, k) in enumerate(idx):
            c = (k * ny + j) * nx + i
            got[r] = F[:, c]
            ref[r] = oracle_face_flux(orc, st, axis, i, j, k)
        scale = np.maximum(np.abs(ref).max(axis=0), 1e-3 * np.abs(ref).max())
        err = (np.abs(got - ref) / scale).max()
        assert err <= tol, (axis, err)
    g.close()


def test_patch_tile_shapes_and_autotune_match_oracle(orc, wb):
    """Patches whose sizes make the cost model pick each of the three x-sweep
    tile shapes (a launch per shape); the same table as one persistent
    launch; then the autotuner's pick: all agree with the oracle patch by
    patch."""
    rng = np.random.default_rng(17)
    dims = [(16, 16, 8), (64, 4, 6), (32, 8, 8), (12, 20, 9)]
    sts = [I.perturbed(*d, seed=40 + n, jump=True) for n, d in enumerate(dims)]
    for s in sts:
        s.dx = s.dy = s.dz = 1.0 / 32
        s.U = I.assemble(*(s.U[0], s.U[1] / s.U[0], s.U[2] / s.U[0], s.U[3] / s.U[0],
                           (s.U[7] - 0.5 * (s.U[1] ** 2 + s.U[2] ** 2 + s.U[3] ** 2) / s.U[0]
                            - 0.5 * (s.U[4] ** 2 + s.U[5] ** 2 + s.U[6] ** 2)) * (s.gamma - 1),
                           s.bx, s.by, s.bz, s.dx, s.dy, s.dz)).U
    dt = 1e-3

    def check(g):
        U, b = g.get_state()
        oU = ob = 0
        for s in sts:
            n = s.U[0].size
            Uo, bxo, byo, bzo = orc.step(ogrid(orc, s), s.U, s.bx, s.by, s.bz, dt, nsteps=2)
            assert rel_err(U[oU:oU + 8 * n].reshape(Uo.shape), Uo).max() <= TOL64
            assert rel_err(b[ob:ob + 3 * n].reshape((3,) + s.shape), np.stack([bxo, byo, bzo])).max() <= TOL64
            oU += 8 * n
            ob += 3 * n

    U0 = np.concatenate([s.U.ravel() for s in sts])
    b0 = np.concatenate([np.stack([s.bx, s.by, s.bz]).ravel() for s in sts])
    g = wb.Grid.from_patches(sts, precision="fp64")
    g.step(dt, 2)
    check(g)
    g.set_tiles(0)
    g.set_state(U0, b0)
    g.step(dt, 2)
    check(g)
    g.set_state(U0, b0)
    ms = g.autotune()
    assert ms.shape == (3, 5) and np.all(ms > 0)
    g.step(dt, 2)
    check(g)
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_every_tile_table_gives_the_same_fluxes(wb, prec):
    """Uneven patches whose cost-model shapes differ per patch: each of the
    autotuner's candidate tables (one persistent launch, one fixed shape
    everywhere, a fixed-shape launch per shape) regroups the same
    interfaces, so the fluxes of every axis agree with the first table to
    rounding, and a step from the same state lands on the same state."""
    sts = I.patch_batch(9, seed=23, lo=12, hi=40)
    g = wb.Grid.from_patches(sts, precision=prec)
    U0, b0 = g.get_state()
    tol = 1e-13 if prec == "fp64" else 2e-6
    ref = None
    for c in range(len(wb.TILE_CANDIDATES)):
        g.set_tiles(c)
        g.set_state(U0, b0)
        F = np.stack([g.face_fluxes(axis) for axis in range(3)])
        g.step(2e-4, 1)
        U1 = g.get_state()[0]
        if ref is None:
            ref = (F, U1)
            continue
        scale = np.abs(ref[0]).max(axis=2, keepdims=True) + 1e-30
        assert (np.abs(F - ref[0]) / scale).max() <= tol, c
        assert np.abs(U1 - ref[1]).max() <= tol * np.abs(ref[1]).max(), c
    with pytest.raises(RuntimeError):
        g.set_tiles(len(wb.TILE_CANDIDATES))
    g.close()


def test_patch_batch_fp32_tracks_fp64(wb):
    """Brio-Wu and turbulence patches of uneven sizes in one FP32 grid stay
    finite and positive and track the FP64 path (L1 per field)."""
    sts = I.patch_batch(12, seed=8, lo=16, hi=32)
    out = {}
    for prec in ("fp64", "fp32"):
        g = wb.Grid.from_patches(sts, precision=prec)
        dt = g.cfl_dt(0.4) if prec == "fp64" else dt
        g.step(dt, 10)
        out[prec] = g.get_state()[0].reshape(-1)
        g.close()
    U64 = np.concatenate([u.reshape(8, -1) for u in np.split(out["fp64"], np.cumsum([8 * s.U[0].size for s in sts])[:-1])], axis=1)
    U32 = np.concatenate([u.reshape(8, -1) for u in np.split(out["fp32"], np.cumsum([8 * s.U[0].size for s in sts])[:-1])], axis=1)
    assert np.isfinite(U32).all() and U32[0].min() > 0
    for f in range(8):
        l1 = np.abs(U32[f] - U64[f]).mean() / max(np.abs(U64[f]).mean(), 1e-30)
        assert l1 < 1e-4, (f, l1)


def test_fp64_weno_z_weights_match_oracle(orc, wb):
    st = I.perturbed(20, 16, 12, seed=77, jump=True)
    g = wb.Grid.from_state(st, precision="fp64", weights="z")
    g.step(2e-3, 2)
    U, bx, by, bz = g.get_state_single()
    g.close()
    nx, ny, nz = st.dims
    og = orc.Grid(nx, ny, nz, st.dx, st.dy, st.dz, st.gamma, 0, 1)
    Uo, bxo, byo, bzo = orc.step(og, st.U, st.bx, st.by, st.bz, 2e-3, nsteps=2)
    assert rel_err(U, Uo).max() <= TOL64
    assert rel_err(np.stack([bx, by, bz]), np.stack([bxo, byo, bzo])).max() <= TOL64
    # and they differ from the Jiang-Shu result
    Uj = orc.step(ogrid(orc, st), st.U, st.bx, st.by, st.bz, 2e-3, nsteps=2)[0]
    assert rel_err(Uj, Uo).max() > 1e3 * TOL64


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_div_b_diagnostic_matches_oracle(orc, wb, precision):
    """wb_div_b against the oracle's face divergence: a field that is not
    solenoidal gives the same maximum; the CT keeps a solenoidal one at
    round-off through steps (also on linked bricks)."""
    from paper_1808_10633_gb300 import bricks

    rng = np.random.default_rng(8)
    st = I.perturbed(20, 16, 12, seed=5)
    og = ogrid(orc, st)
    bad = st.copy()
    bad.bx = bad.bx + 0.01 * rng.standard_normal(bad.bx.shape)
    g = wb.Grid.from_state(bad, precision=precision)
    dmax, bmax = g.div_b()
    g.close()
    ref = np.abs(orc.div_b(og, bad.bx, bad.by, bad.bz)).max()
    tol = 1e-12 if precision == "fp64" else 1e-5
    assert dmax == pytest.approx(ref, rel=tol)
    assert bmax == pytest.approx(max(np.abs(bad.bx).max(), np.abs(bad.by).max(), np.abs(bad.bz).max()), rel=1e-7)
    scale = bmax / min(st.dx, st.dy, st.dz)
    for g in (wb.Grid.from_state(st, precision=precision),
              wb.Grid.from_bricks(st, ([0, 9, 20], [0, 7, 16], [0, 12]), precision=precision)):
        g.step_cfl(0.4, 5)
        d, _ = g.div_b()
        assert d <= (1e-13 if precision == "fp64" else 1e-5) * scale, d / scale
        g.close()


def _degenerate_state(kind, n=(24, 8, 8)):
    """Smooth states whose interface averages sit at the degenerate points
    of the Roe-Balsara normalisation (Sec. 2.1 eigen-system): B_perp = 0
    along x ("bperp0"), the triple point B_perp = 0 with a^2 = B_n^2/rho to
    1e-13 on either side ("triple_hi": a^2 above, "triple_lo": below, so the
    degeneracy rule's choice is decided well above rounding), B_n = 0 along
    x ("bn0"), and no field at all ("hydro").  A density step makes the
    weights nonlinear."""
    nx, ny, nz = n
    x = (np.arange(nx) + 0.5) / nx
    X = np.broadcast_to(x[None, None, :], (nz, ny, nx))
    Y = np.broadcast_to(((np.arange(ny) + 0.5) / ny)[None, :, None], (nz, ny, nx))
    s = np.sin(2 * np.pi * X)
    rho = 1.0 + 0.3 * s + 0.5 * (X > 0.5) + 0.05 * np.cos(2 * np.pi * Y)
    vx, vy, vz = 0.2 * np.cos(2 * np.pi * X), 0.1 * s, -0.1 * np.cos(2 * np.pi * Y)
    gamma = I.GAMMA
    z = np.zeros((nz, ny, nx))
    if kind == "bperp0":
        p, bx, by, bz = 1.0 + 0.1 * s, z + 0.7, z, z
    elif kind in ("triple_hi", "triple_lo"):
        p = z + 1.0
        bx, by, bz = z + np.sqrt(gamma * (1.0 - 1e-13 if kind == "triple_hi" else 1.0 + 1e-13)), z, z
    elif kind == "bn0":
        p, bx, by, bz = 1.0 + 0.1 * s, z, 0.5 + 0.2 * s, z - 0.3
    else:
        p, bx, by, bz = 1.0 + 0.1 * s, z, z, z
    return I.assemble(rho, vx, vy, vz, p, bx, by, bz, 1.0 / nx, 1.0 / ny, 1.0 / nz, gamma=gamma)


@pytest.mark.parametrize("kind", ["bperp0", "triple_hi", "triple_lo", "bn0", "hydro"])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_degenerate_eigen_states_match_oracle(orc, wb, kind, prec, tol):
    """Face fluxes of all three sweeps at the degenerate points of the
    eigenvector normalisation agree with the oracle; the FP32 path takes
    these normalisations in FP64, so it stays at FP32 round-off there too.
    One FP64 step agrees with the oracle's step."""
    st = _degenerate_state(kind)
    nx, ny, nz = st.bx.shape[::-1]
    og = ogrid(orc, st)
    g = wb.Grid.from_state(st, precision=prec)
    for axis in range(3):
        got = g.face_fluxes(axis)
        F8 = orc.face_fluxes(og, st.U, axis).reshape(8, -1)
        t1, t2 = (axis + 1) % 3, (axis + 2) % 3
        ref = np.stack([F8[0], F8[1], F8[2], F8[3], F8[7], F8[4 + t1], F8[4 + t2]])
        floor = 1e-3 * np.abs(ref).max()
        scale = np.maximum(np.abs(ref).max(axis=1, keepdims=True), floor)
        err = (np.abs(got - ref) / scale).max()
        assert err <= tol, (kind, prec, axis, err)
    g.close()
    if prec == "fp64" and kind != "hydro":
        # (with no field, the faces after a step hold only round-off, which
        # compare() would measure against a zero scale)
        compare(orc, wb, st, 1e-3, nsteps=1)
