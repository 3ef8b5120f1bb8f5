"""GPU test of wb_conserved_totals_noalloc, the allocation-free entry point.

It serves callers that cannot call cudaMalloc: code running under another
component's device memory pool, or a loop that cannot take the implicit
device synchronisation of cudaMalloc/cudaFree.  Given the same state in the
caller's device memory, it must agree with wb_conserved_totals (the
allocating entry point) within the totals tolerance used by the other tests,
on two calls in a row: the second call reuses the shared scratch array left
by the first.  This file is collected last so that a run stopping at the
first failure has already run every other test."""
import numpy as np
import pytest

from paper_1808_10633_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wb():
    from paper_1808_10633_gb300 import build, wombat

    build.build()
    return wombat


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_totals_match_allocating_entry_point(wb, prec):
    torch = pytest.importorskip("torch")
    st = I.turbulence(48, seed=21)
    g = wb.Grid.from_state(st, precision=prec)
    ref = g.totals()
    g.close()
    n = st.U[0].size
    # the library's state layout: rho, mx, my, mz, E, bx, by, bz
    fields = np.stack([st.U[0], st.U[1], st.U[2], st.U[3], st.U[7], st.bx, st.by, st.bz])
    dtype = torch.float64 if prec == "fp64" else torch.float32
    dev = torch.from_numpy(fields.reshape(8, n)).to(device="cuda", dtype=dtype).contiguous()
    out = torch.empty(8, dtype=torch.float64, device="cuda")
    dV = st.dx * st.dy * st.dz
    scale = np.abs(st.U).reshape(8, -1).sum(axis=1) * dV
    got = []
    for call in range(2):
        out.fill_(float("nan"))          # a stale or unwritten result cannot pass
        torch.cuda.synchronize()
        wb.conserved_totals_noalloc(dev.data_ptr(), prec, n, dV, out.data_ptr(),
                                    stream=torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        r = out.cpu().numpy()
        assert np.all(np.abs(r - ref) <= 1e-14 * np.maximum(scale, 1e-300)), (call, r, ref)
        got.append(r)
    assert np.array_equal(got[0], got[1])


def test_noalloc_rejects_sizes_beyond_the_maximum(wb):
    torch = pytest.importorskip("torch")
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(wb.WombatError) as e:
        wb.conserved_totals_noalloc(buf.data_ptr(), "fp64", (1 << 34) + 1, 1.0, buf.data_ptr())
    assert e.value.code == wb.WB_EINVAL
    assert "WB_NOALLOC_MAX_CELLS" in str(e.value)
