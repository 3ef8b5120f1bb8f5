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


RESET_SCRIPT = r"""
import ctypes, os, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1808_10633_gb300 import wombat as wb
wb.load()
# the CUDA runtime the library loaded (the same instance, not a second copy)
path = next(l.split()[-1] for l in open("/proc/self/maps") if "libcudart" in l)
rt = ctypes.CDLL(path)
vp = ctypes.c_void_p
rt.cudaMalloc.argtypes = [ctypes.POINTER(vp), ctypes.c_size_t]
rt.cudaMemcpy.argtypes = [vp, vp, ctypes.c_size_t, ctypes.c_int]
rt.cudaFree.argtypes = [vp]
rng = np.random.default_rng(7)
n, dV = 100003, 0.25
for round_ in range(2):
    state = rng.standard_normal(8 * n)
    ds, do = vp(), vp()
    assert rt.cudaMalloc(ctypes.byref(ds), state.nbytes) == 0
    assert rt.cudaMalloc(ctypes.byref(do), 64) == 0
    assert rt.cudaMemcpy(ds, state.ctypes.data, state.nbytes, 1) == 0
    wb.conserved_totals_noalloc(ds.value, "fp64", n, dV, do.value)
    assert rt.cudaDeviceSynchronize() == 0
    out = np.empty(8)
    assert rt.cudaMemcpy(out.ctypes.data, do, 64, 2) == 0
    # state layout rho, mx, my, mz, E, bx, by, bz; totals (rho, m, B, E)
    order = [0, 1, 2, 3, 5, 6, 7, 4]
    ref = state.reshape(8, n).sum(axis=1)[order] * dV
    scale = np.abs(state).reshape(8, n).sum(axis=1)[order] * dV
    assert np.all(np.abs(out - ref) <= 1e-13 * scale), (round_, out, ref)
    rt.cudaFree(ds)
    rt.cudaFree(do)
    if round_ == 0:
        assert rt.cudaDeviceReset() == 0      # ends this process's context only
print("noalloc after reset OK")
"""


def test_noalloc_after_device_reset(wb):
    """A caller (or another library in its process) may reset the device
    between calls: the module is loaded again and the scratch array may move.
    Each call outside stream capture looks its address up again, so the sums
    stay right.  Run in a process of its own (the reset would also end the
    context torch holds in this one)."""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", RESET_SCRIPT, root], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    assert "noalloc after reset OK" in r.stdout
