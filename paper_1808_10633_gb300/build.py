"""Build the CUDA library libwombat_gb300.so in-tree for sm_103a.

nvcc compiles each translation unit of csrc/ in parallel (one -gencode,
arch=compute_103a, code=sm_103a, -lineinfo) and links a shared library next
to this file.  Objects go to _build/ (git-ignored).  The "check" variant
(libwombat_gb300_check.so, objects in _build_check/) is compiled with
-DWB_BOUNDS_CHECK=1: the solver kernels test every index they form and
report a bad one as WB_EINTERNAL instead of touching memory outside an array.
The "tc" variant (libwombat_gb300_tc.so, objects in _build_tc/) runs the
learned-weight networks on the 5th-generation tensor cores (tcgen05) instead
of the per-warp mma.sync form.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libwombat_gb300.so")
VARIANTS = {"release": (OBJ, LIB, []),
            "check": (os.path.join(HERE, "_build_check"), os.path.join(HERE, "libwombat_gb300_check.so"),
                      ["-DWB_BOUNDS_CHECK=1"]),
            "tc": (os.path.join(HERE, "_build_tc"), os.path.join(HERE, "libwombat_gb300_tc.so"),
                   ["-DWB_LEARNED_ENGINE=1"])}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# per-file extra flags: the FP32 sweep uses fast single-precision division
# and square root (FP64 code in that file is unaffected)
EXTRA = {"wb_sweep_f32.cu": ["-use_fast_math"], "wb_sweep_learned.cu": ["-use_fast_math"]}


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libwombat_gb300.so")


def flags(verbose: bool = False):
    f = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]
    # tuning knobs of the kernels (e.g. -DWB_SWEEP_TA_YZ=8), for experiments
    f += os.environ.get("WB_NVCC_FLAGS", "").split()
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) \
        + [os.path.join(ROOT, "include", "wombat_gb300.h"), os.path.abspath(__file__)]


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, jobs: int | None = None,
          variant: str = "release") -> str:
    obj_dir, lib, vflags = VARIANTS[variant]
    if not force and up_to_date(lib):
        return lib
    os.makedirs(obj_dir, exist_ok=True)
    cc = nvcc()
    srcs = _sources()

    def compile_one(src):
        obj = os.path.join(obj_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [cc, *flags(verbose), *vflags, *EXTRA.get(os.path.basename(src), []), "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=jobs or min(len(srcs), os.cpu_count() or 4)) as ex:
        results = list(ex.map(compile_one, srcs))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    objs = [o for o, _ in results]
    tmp = lib + ".tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                variant="check" if "--check" in sys.argv else "release"))
