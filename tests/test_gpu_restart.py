"""Checkpoint/restart and run-to-run determinism through the C ABI.

wb_get_state / wb_init_grid are the checkpoint: the state comes back as FP64
(exact for FP32 storage) and a grid rebuilt from it continues bit for bit
like the grid that kept running.  Two runs of the same inputs give the same
bits (fixed summation orders everywhere, including the CFL maximum and the
conserved totals)."""
import numpy as np
import pytest

from paper_1808_10633_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wb():
    from paper_1808_10633_gb300 import build, wombat

    build.build()
    return wombat


@pytest.mark.parametrize("precision", ["fp64", "fp32", "learned"])
def test_restart_continues_bitwise(wb, precision):
    st = I.add_blasts(I.turbulence(32, seed=12), seed=3, nblast=4, rmin=0.05, rmax=0.1)
    b0 = np.stack([st.bx, st.by, st.bz])

    def grid(U, b):
        g = wb.Grid([st.dims], st.dx, st.dy, st.dz, U, b, gamma=st.gamma, precision=precision)
        if precision == "learned":
            from paper_1808_10633_gb300 import learned as Ln
            g.set_mlp(Ln.init_params(seed=5), 4.0, 0.5)
        return g

    g1 = grid(st.U, b0)
    g1.step_cfl(0.4, 6)
    UA, bA = g1.get_state()
    tA = g1.totals()
    g1.close()
    g2 = grid(st.U, b0)
    g2.step_cfl(0.4, 3)
    Uc, bc = g2.get_state()
    g2.close()
    g3 = grid(Uc, bc)
    g3.step_cfl(0.4, 3)
    UB, bB = g3.get_state()
    tB = g3.totals()
    g3.close()
    assert np.array_equal(UA, UB) and np.array_equal(bA, bB)
    assert np.array_equal(tA, tB)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_runs_are_deterministic(wb, precision):
    sts = I.patch_batch(10, seed=21, lo=12, hi=28)
    out = []
    for _ in range(2):
        g = wb.Grid.from_patches(sts, precision=precision)
        g.autotune()
        g.step_cfl(0.4, 4)
        out.append((g.get_state(), g.totals(), g.cfl_dt(0.4)))
        g.close()
    (U1, b1), t1, d1 = out[0]
    (U2, b2), t2, d2 = out[1]
    assert np.array_equal(U1, U2) and np.array_equal(b1, b2)
    assert np.array_equal(t1, t2) and d1 == d2


def test_fp32_totals_widen_exactly(wb):
    """The FP32 totals widen each value to FP64 with integer operations:
    on values whose FP64 sums are exact in any order (subnormals, signed
    zeros, small-mantissa normals, huge and tiny exponents) the totals equal
    the exact sums."""
    n = 16
    rng = np.random.default_rng(5)
    shape = (n, n, n)
    ints = lambda lo, hi: rng.integers(lo, hi, size=shape).astype(np.float64)
    U = np.zeros((8,) + shape)
    U[0] = ints(-2 ** 20, 2 ** 20) * 2.0 ** -149             # subnormal FP32 values
    U[1] = ints(-1000, 1000) / 1024.0
    U[2] = np.where(rng.random(shape) < 0.5, -0.0, 2.0 ** -126 * ints(-3, 4))
    U[3] = ints(-1000, 1000) * 2.0 ** 100
    U[7] = ints(-2 ** 10, 2 ** 10) * 2.0 ** -140              # subnormal and tiny normal
    b = np.stack([ints(-2 ** 22, 2 ** 22) * 2.0 ** -149, ints(-4, 5) * 1.5, np.full(shape, -0.0)])
    assert np.array_equal(U.astype(np.float32).astype(np.float64), U)
    g = wb.Grid([(n, n, n)], 1.0, 1.0, 1.0, U, b, precision="fp32")
    got = g.totals()
    want = np.array([U[0].sum(), U[1].sum(), U[2].sum(), U[3].sum(),
                     b[0].sum(), b[1].sum(), b[2].sum(), U[7].sum()])
    assert np.array_equal(got, want), (got, want)
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_step_totals_overlap(wb, precision):
    """Per-step totals (second stream inside the step graph) equal the
    explicit totals of the state each step starts from, and leave the
    solution bit for bit unchanged."""
    st = I.turbulence(32, seed=15)
    g1 = wb.Grid.from_state(st, precision=precision)
    g2 = wb.Grid.from_state(st, precision=precision)
    g1.set_step_totals(True)
    g1.step_cfl(0.4, 4)
    g2.step_cfl(0.4, 4)
    t4 = g1.totals()
    g1.step_cfl(0.4, 1)
    g2.step_cfl(0.4, 1)
    assert np.array_equal(g1.step_totals(), t4)
    U1, b1 = g1.get_state()
    U2, b2 = g2.get_state()
    assert np.array_equal(U1, U2) and np.array_equal(b1, b2)
    g1.set_step_totals(False)
    with pytest.raises(wb.WombatError):
        g1.step_totals()
    g1.close()
    g2.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_pinned_host_arrays_in_place(wb, prec):
    """Page-locked host arrays (pinned torch tensors) are read and written in
    place by the import/export kernels, pageable ones staged through a copy:
    both routes move the same bits in FP64 and, on FP32 grids, in FP32."""
    import torch
    st = I.turbulence(20, seed=21)
    g = wb.Grid.from_state(st, precision=prec)
    g.step_cfl(0.4, 2)
    dtypes = (np.float64, np.float32) if prec == "fp32" else (np.float64,)
    for dt in dtypes:
        U0, b0 = g.get_state(dtype=dt)
        tdt = torch.float32 if dt == np.float32 else torch.float64
        Up = torch.empty(U0.size, dtype=tdt).pin_memory()
        bp = torch.empty(b0.size, dtype=tdt).pin_memory()
        g.get_state(Up.numpy(), bp.numpy())
        assert np.array_equal(Up.numpy(), U0) and np.array_equal(bp.numpy(), b0)
        # round trip: pinned in, pageable out, then a step from each route
        h = wb.Grid.from_state(st, precision=prec)
        h.set_state(Up.numpy(), bp.numpy())
        assert np.array_equal(h.get_state(dtype=dt)[0], U0)
        k = wb.Grid.from_state(st, precision=prec)
        k.set_state(U0, b0)
        h.step_cfl(0.4, 1)
        k.step_cfl(0.4, 1)
        assert np.array_equal(h.get_state()[0], k.get_state()[0])
        h.close()
        k.close()
    g.close()


def test_fp32_state_entry_points(wb):
    """wb_set_state_f32 / wb_get_state_f32 move an FP32 grid's state without
    rounding: they agree bit for bit with the FP64 entry points, and a
    restart through them continues bit for bit; FP64 grids refuse them."""
    st = I.turbulence(24, seed=16)
    g = wb.Grid.from_state(st, precision="fp32")
    g.step_cfl(0.4, 2)
    U64, b64 = g.get_state()
    U32, b32 = g.get_state(dtype=np.float32)
    assert U32.dtype == np.float32
    U64r, U32r = U64.reshape(8, -1), U32.reshape(8, -1)
    rows = [0, 1, 2, 3, 7]                     # stored values: exact
    assert np.array_equal(U32r[rows].astype(np.float64), U64r[rows])
    # cell B = mean of two FP32 faces: exact in FP64, correctly rounded in FP32
    assert np.array_equal(U32r[4:7], U64r[4:7].astype(np.float32))
    assert np.array_equal(b32.astype(np.float64), b64)
    h = wb.Grid.from_state(st, precision="fp32")
    h.set_state(U32, b32)
    g.step_cfl(0.4, 2)
    h.step_cfl(0.4, 2)
    assert np.array_equal(g.get_state()[0], h.get_state()[0])
    g.close()
    h.close()
    g = wb.Grid.from_state(st, precision="fp64")
    with pytest.raises(wb.WombatError):
        g.get_state(dtype=np.float32)
    g.close()
