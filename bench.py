"""Benchmark: zone-updates/s per SSP-RK3 step of the WENO5 MHD hot path.

Workload (one GPU): 256^3 periodic decaying turbulence (seeded Gaussian
velocity with per-mode variance |k|^-11/3 for 1<=|k|<=8 at rms Mach 0.5,
log-normal density sigma 0.1, p = 1, B = (0.1,0,0) + solenoidal part at 10%
of the kinetic energy), CFL 0.4.  One step = CFL reduction + dt + three
stages of (x, y, z sweeps, update with constrained transport) + FP64
conserved totals.  The headline value is the FP32-bulk path; the FP64 path,
the FP32 L1 error against FP64 after 20 steps, the end-to-end number through
host buffers, the ALU roofline of the dominant kernel and the CPU oracle are
reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank advances an independent replica on its own
GPU (weak scaling; the path needs no collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "zone-updates/s per RK step at 256^3 (FP32/learned vs FP64) at stated L1 error"
UNIT = "zone-updates/s"

# Algorithmic FP operations of one interface of the sweep kernel (one
# direction, one stage) and of one staged cell, counted from the kernel's
# formulas (add/sub/mul = 1, FMA = 2, div/sqrt = 1): eigen-structure 100,
# interface average 16, central flux 35, differences of the stencil 70,
# their projection 10 x 68, split differences and two phi_N per field
# 7 x 114 (the eps of each smoothness indicator folded into its fused
# multiply-adds, phi_N taken on twice the split differences and halved
# once), back-projection 80.
SWEEP_FLOPS_PER_INTERFACE = 1779
SWEEP_FLOPS_PER_STAGED_CELL = 80

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# FP32 sweep kernels, from one ncu capture of the 256^3 turbulence launch this
# benchmark times (profiles/sweep_traffic_fp32_turbulence256.md); reported
# only at that size and while the sweep sources hash to SWEEP_TRAFFIC_SOURCES.
SWEEP_TRAFFIC_N = 256
SWEEP_TRAFFIC = {"sweep_x": 1180.90e6, "sweep_y": 980.41e6, "sweep_z": 978.70e6}
SWEEP_TRAFFIC_SOURCES = "69dc94dc5fccf3ed"


def sweep_sources_hash() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in ("wb_sweep.cuh", "wb_sweep_f32.cu"):
        with open(os.path.join(ROOT, "paper_1808_10633_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, path: str | None = None):
        self.index = index
        self.path = path
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is None:
            return
        time.sleep(0.2)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        self.lines = [l.strip() for l in out.splitlines() if l.strip()]
        if self.path:
            with open(self.path, "w") as f:
                f.write(self.Q + "\n" + "\n".join(self.lines) + "\n")

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        busy = [s for s in sm if s > 0.5 * max(sm)]
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


_STREAM = None


def cur_stream():
    """The CUDA stream the benchmark's grids run on (a torch stream of its
    own: the legacy default stream has handle 0, which the library reads as
    "make your own stream")."""
    global _STREAM
    if _STREAM is None:
        import torch

        _STREAM = torch.cuda.Stream()
    return _STREAM


def graph_steps_ms(g, k, cfl, world):
    """k steps of grid g (created on cur_stream()) replayed from its step
    graph, timed with CUDA events on that stream between barriers."""
    import torch

    stream = cur_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g.sync()
    barrier(world)
    torch.cuda.synchronize()
    e0.record(stream)
    g.step_cfl(cfl, k)
    e1.record(stream)
    e1.synchronize()
    barrier(world)
    return e0.elapsed_time(e1)


def sweep_units(n):
    """(interfaces, staged cells) per launch of each sweep kernel at n^3."""
    from paper_1808_10633_gb300 import wombat  # noqa: F401  (library must load)
    iface = n ** 3
    # x: tiles of 32 interfaces along the axis stage 37 cells per pencil;
    # y, z: tiles of 16 along the axis stage 21 cells per pencil.
    staged = {"sweep_x": n ** 3 * 37 / 32, "sweep_y": n ** 3 * 21 / 16, "sweep_z": n ** 3 * 21 / 16}
    return iface, staged


def run_native(args, rank, world, local):
    import torch

    from paper_1808_10633_gb300 import inputs, wombat

    n = args.size
    st = inputs.turbulence(n, seed=1808)
    zones = n ** 3
    out = {}
    clocks = Clocks(args.phys_gpu, os.path.join(args.out_dir, f"clocks_rank{rank}.csv") if args.out_dir else None)

    peak32 = wombat.alu_peak_tflops("fp32")
    peak64 = wombat.alu_peak_tflops("fp64") if not args.fp32_only else None

    # ---- FP32 bulk (headline) -------------------------------------------
    # The grid runs on a torch stream, so torch's CUDA events on that stream
    # bracket the step graphs.  A step = CFL dt, three SSP-RK3 stages
    # (sweeps, EMFs, updates) and the FP64 conserved totals of its start
    # state (on a second stream inside the step graph).
    stream = cur_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed_steps(g, k):
        g.sync()
        barrier(world)
        torch.cuda.synchronize()
        ev0.record(stream)
        g.step_cfl(args.cfl, k)
        ev1.record(stream)
        ev1.synchronize()
        torch.cuda.synchronize()
        barrier(world)
        return ev0.elapsed_time(ev1)

    g32 = wombat.Grid.from_state(st, precision="fp32", stream=stream.cuda_stream)
    g32.set_step_totals(True)
    g32.step_cfl(args.cfl, args.warmup)
    with clocks:
        tot_ms = timed_steps(g32, args.steps)
        # FP64 path inside the same clock window
        g64 = None
        if not args.fp32_only:
            g64 = wombat.Grid.from_state(st, precision="fp64", stream=stream.cuda_stream)
            g64.set_step_totals(True)
            g64.step_cfl(args.cfl, 1)
            k64 = max(2, args.steps // 4)
            tot64 = timed_steps(g64, k64)
    secs = max_over_ranks(tot_ms / 1e3, world)
    value = world * zones * args.steps / secs
    if g64 is not None:
        secs64 = max_over_ranks(tot64 / 1e3, world)
        value64 = world * zones * k64 / secs64
    clk = clocks.summary()
    step_totals = g32.step_totals()

    # per-kernel split of the same step (CUDA events around every launch,
    # kernels serialised, totals on the same stream)
    g32.sync()
    prof_ms, kms, kcnt = g32.step_profiled(args.cfl, args.steps, with_totals=True)
    if g64 is not None:
        g64.sync()
        _, kms64, kcnt64 = g64.step_profiled(args.cfl, k64, with_totals=True)

    def roofline(kms_, kcnt_, peak_tflops, label):
        cls = max((k for k in ("sweep_x", "sweep_y", "sweep_z")), key=lambda k: kms_[k])
        per_launch_ms = kms_[cls] / max(kcnt_[cls], 1)
        iface, staged = sweep_units(n)
        flops = iface * SWEEP_FLOPS_PER_INTERFACE + staged[cls] * SWEEP_FLOPS_PER_STAGED_CELL
        achieved = flops / (per_launch_ms * 1e-3) / 1e12
        traffic = None
        if label == "float" and n == SWEEP_TRAFFIC_N and sweep_sources_hash() == SWEEP_TRAFFIC_SOURCES:
            traffic = SWEEP_TRAFFIC[cls]
        alg_bytes = iface * 4 * (8 + 7 + (3 if cls == "sweep_x" else 0)) * (1 if label == "float" else 2)
        return {"kernel": f"sweep_kernel_fixed<{label},{'xyz'[('sweep_x','sweep_y','sweep_z').index(cls)]}>",
                "bound": "alu", "achieved": round(achieved, 3), "peak": round(peak_tflops, 3),
                "unit": "TFLOP/s", "frac": round(achieved / peak_tflops, 4), "traffic": traffic,
                "traffic_note": None if traffic is None else
                f"ncu dram__bytes_read.sum + dram__bytes_write.sum of this launch at {n}^3 (bytes per launch)",
                "traffic_vs_algorithmic": None if traffic is None else round(traffic / alg_bytes, 4),
                "algorithmic_bytes_per_launch": alg_bytes,
                "flops_per_launch": flops, "ms_per_launch": round(per_launch_ms, 4),
                "peak_source": "measured FMA throughput (wb_alu_peak) on this GPU"}

    rf32 = roofline(kms, kcnt, peak32, "float")
    rf64 = roofline(kms64, kcnt64, peak64, "double") if g64 is not None else None

    # ---- FP32 vs FP64 L1 error after l1_steps fixed-dt steps (rank 0) ----
    l1 = None
    if rank == 0 and args.l1_steps > 0 and g64 is not None:
        g64.set_state(st.U, np.stack([st.bx, st.by, st.bz]))
        g32.set_state(st.U, np.stack([st.bx, st.by, st.bz]))
        dt = g64.cfl_dt(args.cfl)
        g64.step(dt, args.l1_steps)
        g32.step(dt, args.l1_steps)
        U64, _ = g64.get_state()
        U32, _ = g32.get_state()
        U64 = U64.reshape(8, -1)
        U32 = U32.reshape(8, -1)
        names = ["rho", "mx", "my", "mz", "Bx", "By", "Bz", "E"]
        l1 = {}
        for f, nm in enumerate(names):
            d = np.abs(U32[f] - U64[f])
            l1[nm] = {"l1_rel": float(d.mean() / max(np.abs(U64[f]).mean(), 1e-300)),
                      "linf_rel": float(d.max() / max(np.abs(U64[f]).max(), 1e-300))}
    if g64 is not None:
        g64.close()

    # ---- 4096 batched uneven periodic patches (edges 16-64) ------------------
    patches = None
    if args.patches > 0:
        patches = run_patches(args, world)

    # ---- the same world as linked bricks ------------------------------------
    linked = None
    if not args.no_linked:
        linked = run_linked(args, st, world)

    # ---- 512^3 turbulence + blasts, sweep kernels only ----------------------
    large = None
    if args.large_size > 0:
        large = run_large(args, world)

    # ---- learned weights on 256^3 turbulence + blasts ----------------------
    learned = None
    if not args.no_learned:
        args.sm_mhz = clk.get("sm_mhz")
        learned = run_learned(args, st, world, peak32)

    # ---- end to end through the ABI with pinned host buffers --------------
    e2e = None
    if not args.no_e2e:
        # the FP32 grid's own precision at the ABI (wb_set_state_f32 /
        # wb_get_state_f32): exact, half the bytes of the FP64 entry points
        Uh = torch.from_numpy(np.ascontiguousarray(st.U, dtype=np.float32).ravel()).pin_memory()
        bh = torch.from_numpy(np.stack([st.bx, st.by, st.bz]).astype(np.float32).ravel()).pin_memory()
        Uo = torch.empty(8 * zones, dtype=torch.float32).pin_memory()
        bo = torch.empty(3 * zones, dtype=torch.float32).pin_memory()
        for _ in range(1):
            g32.set_state(Uh, bh)
            g32.step_cfl(args.cfl, 1)
            g32.get_state(Uo, bo)
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            g32.set_state(Uh, bh)
            g32.step_cfl(args.cfl, 1)
            g32.get_state(Uo, bo)
        el = time.perf_counter() - t0
        barrier(world)
        el = max_over_ranks(el, world)
        # bytes over the host link: the import reads rho, m, E of U and the
        # three face arrays of b (U's cell-centred B follows from the faces);
        # the export writes all of U and b
        e2e = {"value": world * zones * args.steps / el, "unit": UNIT,
               "h2d_bytes_per_step": int(8 * zones * 4),
               "d2h_bytes_per_step": int(Uo.numel() * 4 + bo.numel() * 4),
               "path": "wb_set_state_f32(pinned) + wb_step_cfl(1) + wb_get_state_f32(pinned), "
                       "the whole state in and out every step"}
    g32.close()

    launches_per_step = sum(kcnt.values()) / args.steps
    out.update({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded turbulence generator, no dataset)",
        "config": {"workload": f"decaying MHD turbulence {n}^3 periodic, SSP-RK3, CFL {args.cfl}, "
                               "WENO5-JS characteristic sweeps + CT",
                   "grid": [n, n, n], "precision": "fp32-bulk (fp64 islands)",
                   "l2": "inputs larger than L2 (state 8 x 64 MiB fp32 + fluxes)",
                   "parallelism": f"replicas x{world}"},
        # kernels in the timed region: per step the profiled classes, with the
        # totals class counting its two kernels
        "gpu_launches": int(sum(kcnt.values()) + kcnt.get("totals", 0)),
        "launches_per_step": launches_per_step,
        "profiled_ms_per_step": prof_ms / args.steps,
        "kernel_ms_per_step": {k: v / args.steps for k, v in kms.items()},
        "step_totals_last": step_totals.tolist(),
        "roofline": rf32,
        "fp64": None if g64 is None else
                {"value": value64, "unit": UNIT, "ms_per_step": secs64 * 1e3 / k64, "steps": k64,
                 "kernel_ms_per_step": {k: v / k64 for k, v in kms64.items()}, "roofline": rf64},
        "speedup_fp32_over_fp64": (value / value64) if g64 is not None else None,
        "fp32_vs_fp64_after_steps": args.l1_steps if l1 else 0,
        "fp32_error_vs_fp64": l1,
        "alu_peak_tflops": {"fp32": peak32, "fp64": peak64},
        "clocks": clk,
        "e2e": e2e,
        "learned": learned,
        "patches": patches,
        "large": large,
        "linked": linked,
    })
    # the other legs' headline rates in one short object at the end of the line
    out["legs"] = {
        "fp64": out["fp64"]["value"] if out["fp64"] else None,
        "e2e": e2e["value"] if e2e else None,
        "learned": learned["value"] if learned else None,
        "learned_gain_vs_js": learned.get("gain_vs_js") if learned else None,
        "patches": patches["value"] if patches else None,
        "large_whole_step": large.get("value_whole_step") if large else None,
        "linked": linked["value"] if linked else None,
    }
    return out


def run_patches(args, world):
    """Independent periodic patches, edges log-uniform in [16, 64] (aspect
    <= 2), each a rotated Brio-Wu tube or a turbulence state; FP32, per-patch
    tile shapes (a launch per shape and sweep axis), then autotuned."""
    import torch

    from paper_1808_10633_gb300 import inputs, wombat

    t0 = time.perf_counter()
    sts = inputs.patch_batch(args.patches, seed=1808)
    t_gen = time.perf_counter() - t0
    cells = sum(s.U[0].size for s in sts)
    g = wombat.Grid.from_patches(sts, precision="fp32", stream=cur_stream().cuda_stream)
    g.set_step_totals(True)
    g.step_cfl(args.cfl, args.warmup)
    tot0 = graph_steps_ms(g, args.steps, args.cfl, world)      # cost-model tiles
    tune = g.autotune()
    g.step_cfl(args.cfl, 2)
    tot = graph_steps_ms(g, args.steps, args.cfl, world)
    secs = max_over_ranks(tot / 1e3, world)
    g.sync()
    _, kms, kcnt = g.step_profiled(args.cfl, args.steps, with_totals=True)
    g.close()
    return {"workload": f"{args.patches} periodic patches, edges log-uniform in [16,64], "
                        "Brio-Wu or turbulence, FP32", "cells": int(cells),
            "value": world * cells * args.steps / secs, "unit": UNIT,
            "ms_per_step": secs * 1e3 / args.steps,
            "ms_per_step_cost_model_tiles": tot0 / args.steps,
            "kernel_ms_per_step": {k: v / args.steps for k, v in kms.items()},
            "autotune_ms": {"x": tune[0].tolist(), "y": tune[1].tolist(), "z": tune[2].tolist(),
                            "columns": list(wombat.TILE_CANDIDATES)},
            "generate_s": t_gen}


def run_linked(args, st, world):
    """The headline turbulence world cut into 4 x 4 x 4 uneven bricks that
    read their neighbours' cells in place (FP32, same steps)."""
    import torch

    from paper_1808_10633_gb300 import wombat

    n = args.size
    cut = lambda f: [0] + [int(round(n * x)) for x in f] + [n]
    cuts = (cut([0.22, 0.47, 0.74]), cut([0.27, 0.5, 0.77]), cut([0.24, 0.53, 0.76]))
    g = wombat.Grid.from_bricks(st, cuts, precision="fp32", stream=cur_stream().cuda_stream)
    g.set_step_totals(True)
    g.step_cfl(args.cfl, args.warmup)
    tot0 = graph_steps_ms(g, args.steps, args.cfl, world)      # cost-model tiles
    tune = g.autotune()
    g.step_cfl(args.cfl, 2)
    tot = graph_steps_ms(g, args.steps, args.cfl, world)
    secs = max_over_ranks(tot / 1e3, world)
    g.sync()
    _, kms, kcnt = g.step_profiled(args.cfl, args.steps, with_totals=True)
    g.close()
    return {"workload": f"turbulence {n}^3 as 64 linked bricks (cuts {cuts}), FP32",
            "value": world * n ** 3 * args.steps / secs, "unit": UNIT,
            "ms_per_step": secs * 1e3 / args.steps, "ms_per_step_cost_model_tiles": tot0 / args.steps,
            "kernel_ms_per_step": {k: v / args.steps for k, v in kms.items()},
            "autotune_ms": {"x": tune[0].tolist(), "y": tune[1].tolist(), "z": tune[2].tolist(),
                            "columns": list(wombat.TILE_CANDIDATES)}}


def run_large(args, world):
    """512^3 turbulence with 64 blast spheres (p x100, radii 0.02-0.05) in
    FP32 with FP64 islands; the rate counts the three sweep kernels only."""
    import torch

    from paper_1808_10633_gb300 import inputs, wombat

    n = args.large_size
    t0 = time.perf_counter()
    st = inputs.add_blasts(inputs.turbulence(n, seed=1808), seed=1808, nblast=64)
    t_gen = time.perf_counter() - t0
    g = wombat.Grid.from_state(st, precision="fp32", stream=cur_stream().cuda_stream)
    g.set_step_totals(True)
    blast_cells = st.meta.get("blast_cells")
    del st
    steps = max(2, args.large_steps)
    g.step_cfl(args.cfl, args.warmup)
    tot = graph_steps_ms(g, steps, args.cfl, world)
    secs = max_over_ranks(tot / 1e3, world)
    g.sync()
    # the sweeps' own time from CUDA events around each launch
    _, kms, kcnt = g.step_profiled(args.cfl, steps, with_totals=True)
    sweep_ms = sum(kms[k] for k in ("sweep_x", "sweep_y", "sweep_z"))
    sweep_s = max_over_ranks(sweep_ms / 1e3, world)
    try:
        finite = bool(np.isfinite(g.totals()).all())
    except wombat.WombatError:
        finite = False
    g.close()
    zones = n ** 3
    return {"workload": f"turbulence {n}^3 + 64 blast spheres (p x100, r 0.02-0.05), FP32 with FP64 islands",
            "value_sweeps_only": world * zones * steps / sweep_s,
            "value_whole_step": world * zones * steps / secs, "unit": UNIT, "steps": steps,
            "sweep_ms_per_step": sweep_s * 1e3 / steps,
            "kernel_ms_per_step": {k: v / steps for k, v in kms.items()},
            "blast_cells": blast_cells, "finite_after": finite,
            "generate_s": t_gen}


def bf16_peak_tflops():
    """Measured dense BF16 tensor peak of this GPU (sustained, for a kernel
    inside a long step) from MEASURED_PEAKS.json, else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops_sustained"]), "measured (MEASURED_PEAKS.json, sustained)"
    except (OSError, KeyError, ValueError):
        return 1700.0, "fallback (1.7 PFLOP/s sustained)"


# Special-function (MUFU) operations per interface of the learned sweep: the
# GELU takes one hardware tanh per BF16 pair (14 network evaluations x 2
# hidden layers x 16 pairs), the softmax three exponentials and a reciprocal
# per evaluation, the input normalisation one reciprocal per evaluation.
LEARNED_SFU_PER_INTERFACE = 14 * 2 * 16 + 14 * 4 + 14
SFU_OPS_PER_CLK_PER_SM = 16          # 4 per SM sub-partition


def learned_roofline(n, cls, ms_launch, mlp_flops, peak32, sm_mhz, nsm):
    """Roofline time of one learned sweep launch: the Jiang-Shu part of the
    sweep at the FP32 FMA peak plus the networks at the BF16 tensor peak
    (additive), against the measured launch time; beside it the same with
    the GELU's special-function operations at the MUFU rate (unit count x
    the SM clock seen during the run)."""
    iface, staged = sweep_units(n)
    alu_flops = iface * SWEEP_FLOPS_PER_INTERFACE + staged[cls] * SWEEP_FLOPS_PER_STAGED_CELL
    bf16, src = bf16_peak_tflops()
    t_roof = alu_flops / (peak32 * 1e12) + mlp_flops / (bf16 * 1e12)
    sfu_rate = SFU_OPS_PER_CLK_PER_SM * nsm * sm_mhz * 1e6
    t_sfu = iface * LEARNED_SFU_PER_INTERFACE / sfu_rate
    return {"bound": "alu+tensor", "ms_per_launch": round(ms_launch, 4),
            "ms_at_peaks": round(t_roof * 1e3, 4), "frac": round(t_roof * 1e3 / ms_launch, 4),
            "fp32_peak_tflops": round(peak32, 3), "bf16_peak_tflops": bf16, "bf16_peak_source": src,
            "sfu_ms_at_peak": round(t_sfu * 1e3, 4),
            "frac_with_sfu": round((t_roof + t_sfu) * 1e3 / ms_launch, 4),
            "sfu_peak_source": f"{SFU_OPS_PER_CLK_PER_SM} MUFU ops/clk/SM x {nsm} SMs x {sm_mhz:.0f} MHz"}


def _l1(U, ref):
    names = ["rho", "mx", "my", "mz", "Bx", "By", "Bz", "E"]
    U = U.reshape(8, -1)
    ref = ref.reshape(8, -1)
    return {nm: float(np.abs(U[f] - ref[f]).mean() / max(np.abs(ref[f]).mean(), 1e-300))
            for f, nm in enumerate(names)}


def run_learned(args, st, world, peak32):
    """Learned weights (BF16 tensor-core MLP per characteristic field, Jiang-
    Shu where the detectors fire) on the turbulence field with 64 blast
    spheres.  The networks are trained here, by the library's own harvest,
    forward/backward and Adam kernels, on faces of a 64^3 turbulence state."""
    import torch

    from paper_1808_10633_gb300 import inputs, learned as Ln, wombat

    t0 = time.perf_counter()
    rec = Ln.harvest(inputs.turbulence(64, seed=1808), 20000, seed=5)
    t_h = time.perf_counter() - t0
    params, hist = Ln.train(rec, steps=1500, batch=4096, lr=2e-3, lam=1e-3, seed=6)
    t_t = time.perf_counter() - t0 - t_h
    st5 = inputs.add_blasts(st, seed=1808, nblast=64)
    n = args.size
    zones = n ** 3
    gl = wombat.Grid.from_state(st5, precision="learned", stream=cur_stream().cuda_stream)
    gl.set_mlp(params, 4.0, 0.5, smooth=args.smooth)
    gl.set_step_totals(True)
    gl.step_cfl(args.cfl, args.warmup)
    gl.learned_stats(reset=True)
    tot = graph_steps_ms(gl, args.steps, args.cfl, world)
    secs = max_over_ranks(tot / 1e3, world)
    value = world * zones * args.steps / secs
    fired, decisions = gl.learned_stats(reset=True)
    gl.sync()
    _, kms, kcnt = gl.step_profiled(args.cfl, args.steps, with_totals=True)
    # MLP work: 14 evaluations (7 fields x 2 sides) of 2*(6*32+32*32+32*3) flops per interface
    mlp_flops = 14 * 2 * (6 * 32 + 32 * 32 + 32 * 3) * zones
    cls = max(("sweep_x", "sweep_y", "sweep_z"), key=lambda k: kms[k])
    ms_l = kms[cls] / max(kcnt[cls], 1)
    props = torch.cuda.get_device_properties(0)
    sm_mhz = float(getattr(args, "sm_mhz", None) or 2070.0)
    res = {"workload": f"turbulence {n}^3 + 64 blast spheres (p x100, r 0.02-0.05), learned weights "
                       f"(smoothness gate {args.smooth})",
           "value": value, "unit": UNIT, "ms_per_step": secs * 1e3 / args.steps,
           "kernel_ms_per_step": {k: v / args.steps for k, v in kms.items()},
           "train": {"records": int(rec.shape[0]), "unflagged": int((rec[:, 11] == 0).sum()),
                     "steps": 1500, "harvest_s": t_h, "train_s": t_t,
                     "loss_first": float(hist[:20].mean()), "loss_last": float(hist[-20:].mean())},
           "sweep_mlp_tflops": mlp_flops / (ms_l * 1e-3) / 1e12,
           "roofline": learned_roofline(n, cls, ms_l, mlp_flops, peak32, sm_mhz, props.multi_processor_count),
           "js_weight_rate": fired / max(decisions, 1), "weight_decisions": decisions}
    # what the networks gain: Alfven-wave L1 error against the exact solution
    gain = Ln.alfven_gain(params, Ns=(16, 32, 64), smooth=args.smooth)
    res["gain_vs_js"] = {str(N): round(g["vs_js"], 4) for N, g in gain.items()}
    res["gain_vs_weno_z"] = {str(N): round(g["vs_weno_z"], 4) for N, g in gain.items()}
    res["gain_l1"] = {str(N): {k: g[k] for k in ("learned", "js", "weno_z", "js_decisions")}
                      for N, g in gain.items()}
    res["gain_workload"] = ("circularly polarised Alfven wave, amplitude 0.1, N x 1 x 1, t = 0.2, "
                            "L1 of B_y against the exact solution; ratios learned / Jiang-Shu and "
                            "learned / WENO-Z, all FP32")
    if args.l1_steps > 0:
        nst = max(1, args.l1_steps // 2)
        b5 = np.stack([st5.bx, st5.by, st5.bz])
        g64 = wombat.Grid.from_state(st5, precision="fp64")
        dt = g64.cfl_dt(args.cfl)
        g64.step(dt, nst)
        U64, _ = g64.get_state()
        g64.close()
        g32 = wombat.Grid.from_state(st5, precision="fp32")
        g32.step(dt, nst)
        U32, _ = g32.get_state()
        g32.close()
        gl.set_state(st5.U, b5)
        gl.step(dt, nst)
        Ul, _ = gl.get_state()
        res["error_vs_fp64_after_steps"] = nst
        res["l1_rel_vs_fp64"] = {"learned": _l1(Ul, U64), "fp32_js": _l1(U32, U64)}
        # the plain turbulence workload (no blasts), same steps
        b2 = np.stack([st.bx, st.by, st.bz])
        g64 = wombat.Grid.from_state(st, precision="fp64")
        dt2 = g64.cfl_dt(args.cfl)
        g64.step(dt2, nst)
        U64t, _ = g64.get_state()
        g64.close()
        gl.set_state(st.U, b2)
        gl.step(dt2, nst)
        Ult, _ = gl.get_state()
        res["l1_rel_vs_fp64_turbulence"] = _l1(Ult, U64t)
    gl.close()
    return res


def oracle_sample(seconds: float, n: int, cfl: float):
    """Time the FP64 CPU oracle on an n^3 sample of the same workload until
    `seconds` of wall time have elapsed (at least one step)."""
    import oracle
    from paper_1808_10633_gb300 import inputs

    st = inputs.turbulence(n, seed=1808)
    g = oracle.Grid(n, n, n, st.dx, st.dy, st.dz, st.gamma)
    U, bx, by, bz = st.U, st.bx, st.by, st.bz
    steps = 0
    t0 = time.perf_counter()
    while True:
        U, bx, by, bz, _ = oracle.step_cfl(g, U, bx, by, bz, cfl, nsteps=1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return n ** 3 * steps / el, steps, el, oracle.num_threads()


def run_reference(args, rank, world):
    """Reference arm: the paper publishes no code, so the reference program is
    the FP64 CPU oracle of the same scheme, timed on the host cores, each step
    one SSP-RK3 step (with its CFL dt) of an n^3 sample of the workload."""
    if rank != 0:
        return None
    import oracle
    from paper_1808_10633_gb300 import inputs

    n = args.ref_size
    st = inputs.turbulence(n, seed=1808)
    g = oracle.Grid(n, n, n, st.dx, st.dy, st.dz, st.gamma)
    U, bx, by, bz = st.U, st.bx, st.by, st.bz
    for _ in range(args.warmup):
        U, bx, by, bz, _ = oracle.step_cfl(g, U, bx, by, bz, args.cfl, nsteps=1)
    t0 = time.perf_counter()
    U, bx, by, bz, _ = oracle.step_cfl(g, U, bx, by, bz, args.cfl, nsteps=args.steps)
    tot = time.perf_counter() - t0
    cores = oracle.num_threads()
    value = n ** 3 * args.steps / tot
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded turbulence generator, no dataset)",
            "config": {"workload": f"decaying MHD turbulence, FP64 CPU oracle on a {n}^3 sample of the "
                                   f"{args.size}^3 workload, SSP-RK3, CFL {args.cfl}",
                       "grid": [n, n, n]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} SSP-RK3 steps of a {n}^3 periodic turbulence sample"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--ref-size", type=int, default=64)
    ap.add_argument("--cfl", type=float, default=0.4)
    ap.add_argument("--l1-steps", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-weights leg")
    ap.add_argument("--no-linked", action="store_true", help="skip the linked-bricks leg")
    ap.add_argument("--large-size", type=int, default=512,
                    help="edge of the turbulence + blasts leg timed on its sweeps (0: skip)")
    ap.add_argument("--large-steps", type=int, default=10)
    ap.add_argument("--patches", type=int, default=4096,
                    help="patch count of the batched-patch leg (0: skip)")
    ap.add_argument("--smooth", type=float, default=1.03,
                    help="smoothness gate of the learned weights (wb_set_mlp_gate)")
    ap.add_argument("--fp32-only", action="store_true",
                    help="time the FP32 step only (no FP64 leg, L1 comparison, e2e or CPU baseline)")
    ap.add_argument("--out-dir", default=os.environ.get("WB_BENCH_OUT"),
                    help="directory for the clock samples (CSV); none by default")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.fp32_only:
        args.no_e2e = args.no_cpu = args.no_learned = True
        args.patches = 0
        args.l1_steps = 0
    rank, world, local = dist_env()
    # one GPU per rank: restrict this process to its GPU before CUDA starts,
    # so that torch and the library see the same device 0
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    ids = vis.split(",") if vis else None
    args.phys_gpu = int(ids[local]) if ids and local < len(ids) and ids[local].isdigit() else local
    if args.impl == "native":
        os.environ["CUDA_VISIBLE_DEVICES"] = str(args.phys_gpu)
    if args.out_dir:
        os.makedirs(args.out_dir, exist_ok=True)

    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res), flush=True)
        return

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    from paper_1808_10633_gb300 import build
    build.build()
    res = run_native(args, rank, world, local)
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle

        v, s, el, cores = oracle_sample(args.cpu_seconds, args.ref_size, args.cfl)
        res["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"{s} SSP-RK3 steps of a {args.ref_size}^3 periodic turbulence "
                                         f"sample of the same generator, {el:.1f} s wall"}
        # the same oracle on one host core (a 32^3 sample, a few seconds)
        oracle.set_num_threads(1)
        v1, s1, el1, _ = oracle_sample(min(5.0, args.cpu_seconds), 32, args.cfl)
        oracle.set_num_threads(cores)
        res["cpu_baseline"]["single_core"] = {"value": v1, "unit": UNIT, "cores": 1,
                                              "sample": f"{s1} steps of a 32^3 sample, {el1:.1f} s wall"}
    if rank == 0:
        if "legs" in res:
            res["legs"] = res.pop("legs")          # keep the short summary last
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
