"""The training targets of the learned weights: exact face reconstructions
of periodic point values (paper_1808_10633_gb300.learned).  Checked against
the closed form for a sinusoid and against the fifth-order upwind
reconstruction, which must converge to them at fifth order."""
import os

import numpy as np

from paper_1808_10633_gb300 import learned as Ln

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "weno5_linear.txt")


def test_sinusoid_closed_form():
    for N in (16, 32, 64):
        x = (np.arange(N) + 0.5) / N
        for k in (1, 3, 5):
            f = np.cos(2 * np.pi * k * x) + 0.3 * np.sin(2 * np.pi * 2 * x)
            h = Ln.face_reconstruction(f[None, :], -1)[0]
            th1, th2 = 2 * np.pi * k / N, 2 * np.pi * 2 / N
            xf = x + 0.5 / N
            ref = (th1 / 2) / np.sin(th1 / 2) * np.cos(2 * np.pi * k * xf) \
                + 0.3 * (th2 / 2) / np.sin(th2 / 2) * np.sin(2 * np.pi * 2 * xf)
            assert np.abs(h - ref).max() < 1e-12


def test_upwind5_converges_to_exact_face_values_at_fifth_order():
    num = None
    for line in open(GOLDEN):
        if line.startswith("upwind5_num"):
            num = np.array([float(v) for v in line.split()[1:]]) / 60.0
    errs = []
    for N in (32, 64, 128):
        x = (np.arange(N) + 0.5) / N
        f = np.exp(np.sin(2 * np.pi * x))
        h = Ln.face_reconstruction(f[None, :], -1)[0]
        up = sum(num[m] * np.roll(f, 2 - m) for m in range(5))   # f_{i-2..i+2}
        errs.append(np.abs(up - h).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders.min() > 4.7, (errs, orders)

