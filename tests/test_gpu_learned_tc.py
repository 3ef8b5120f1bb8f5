"""The learned-weight suites re-run on the tensor-core build of the library.

The "tc" variant evaluates the per-field networks with tcgen05.mma (BF16
operands in shared memory, FP32 accumulators in tensor memory, one issuing
thread per block) instead of the per-warp mma.sync form of the default
build.  The learned-sweep parity cases against the FP64 reference network
(linear and random networks, the smoothness gate, the detector fallback),
the gain on the Alfven wave, positivity on blasts, the detector log, linked
bricks and restarts pass on it unchanged."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_learned_suites_pass_on_tensor_core_build():
    from paper_1808_10633_gb300 import build

    lib = build.build(variant="tc")
    env = dict(os.environ, WB_LIBRARY=lib)
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
           os.path.join(ROOT, "tests", "test_gpu_learned.py"),
           os.path.join(ROOT, "tests", "test_gpu_linked.py"),
           os.path.join(ROOT, "tests", "test_gpu_restart.py"),
           "-k", "learned or detector"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert "passed" in r.stdout
