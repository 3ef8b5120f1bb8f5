"""Run a grid to a time or a step count and log one JSON line per report.

Each line holds the step count, simulated time, the last dt (CFL rule, taken
on the device), the FP64 conserved totals (rho, mx, my, mz, Bx, By, Bz, E
summed over cells times the cell volume), the face divergence of b (maximum,
and relative to max|b| / min(dx, dy, dz)), the detector fire rate of a
learned grid, and zone-updates/s over the steps since the previous line.
Everything is read through the library's own calls; nothing is computed
here beyond ratios.
"""
from __future__ import annotations

import json
import time
from typing import Callable, Optional

from . import wombat


def run(grid: "wombat.Grid", t_end: Optional[float] = None, nsteps: Optional[int] = None,
        cfl: float = 0.4, every: int = 1, emit: Callable[[str], None] = print,
        hmin: Optional[float] = None) -> dict:
    """Advance `grid` until `t_end` (the last step shortened to land on it)
    or for `nsteps` steps, emitting a JSON line every `every` steps and at
    the end.  `hmin` is the smallest cell size (for the relative div b).
    Returns the last record."""
    if t_end is None and nsteps is None:
        raise ValueError("give t_end or nsteps")
    learned = grid.precision == "learned"
    if learned:
        grid.learned_stats(reset=True)
    t, step, rec = 0.0, 0, {}
    t0 = time.perf_counter()
    last_step, last_t = 0, t0
    while True:
        if nsteps is not None and step >= nsteps:
            break
        if t_end is not None and t >= t_end * (1 - 1e-14):
            break
        dt = grid.cfl_dt(cfl)
        if t_end is not None:
            dt = min(dt, t_end - t)
        grid.step(dt, 1)
        t += dt
        step += 1
        done = (nsteps is not None and step >= nsteps) or (t_end is not None and t >= t_end * (1 - 1e-14))
        if step % every == 0 or done:
            totals = grid.totals()
            dmax, bmax = grid.div_b()
            now = time.perf_counter()
            rec = {"step": step, "t": t, "dt": dt, "totals": totals.tolist(), "div_b_max": dmax,
                   "div_b_rel": dmax * hmin / bmax if (hmin and bmax > 0) else None,
                   "zone_updates_per_s": grid.ncells * (step - last_step) / max(now - last_t, 1e-12)}
            if learned:
                fired, decisions = grid.learned_stats(reset=True)
                rec["detector_fire_rate"] = fired / max(decisions, 1)
            emit(json.dumps(rec))
            last_step, last_t = step, now
    return rec
