"""Time-stepped use of the field solve in a toy particle-mesh loop.

Each step (Sec. 3.3, step 2: a step's solve starts from the previous step's
solution): solve the f(R) field for the current particles, form the potential
of matter plus effective mass on the PM grid (Sec. 2.4, Eq. (30)), take its
force at the particles and move them by one leapfrog kick-drift.  All of it
runs in the library (mgfr_solve_particles, mgfr_pm_accel, mgfr_kick_drift);
this module only sequences the calls and records what each start costs.

At every step the same particle configuration is solved from a zero start,
from the previous step's solution on the base level (MGFR_START_PREVIOUS, the
paper's step list), from the previous step's solution on every level where
its octs persist (MGFR_START_PREVIOUS_ALL) and, when a network is given, from
the learned start; only the previous-start solve's context drives the
trajectory.  The integrator is a toy: the kick is chosen once so
that the fastest particle moves about `move_cells` base cells over the run.
"""
from __future__ import annotations

from . import mgfr


def _cycles(st: dict) -> int:
    """V-cycles of every level: base (FP32 cycles and FP64 outer iterations)
    plus the refined levels' cycles."""
    return int(st["vcycles"] + st["outer_iters"] + sum(st["level_iters"][1:st["n_levels"]]))


def run(pos, N_base: int, box: float, steps: int, fr0: float, max_level: int,
        precision: int = mgfr.PREC_MIXED, a: float = 1.0, net_path: str | None = None,
        move_cells: float = 1.0, device: int = 0):
    """Run the loop from positions `pos` ([Np, 3] CUDA FP64, modified in
    place).  Returns one dict per step with, per start ('zero', 'previous',
    'previous_all', 'learned' if net_path), the V-cycles of all levels and the
    device time of the solve (ms), and the largest relative difference of the
    base f_R between the starts."""
    import torch
    kw = dict(fr0_abs=fr0, precision=precision, max_level=max_level)
    warm = mgfr.Solver(device, **kw)
    zero = mgfr.Solver(device, **kw)
    wall = mgfr.Solver(device, start=mgfr.START_PREVIOUS_ALL, **kw)
    lrn = None
    if net_path:
        lrn = mgfr.Solver(device, start=mgfr.START_LEARNED, **kw)
        lrn.unet_load(net_path)
    vel = torch.zeros_like(pos)
    kick = None
    rows = []
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(s, **k):
        ev[0].record()
        out = s.solve_particles(pos, N_base, box, a, want_acc=False, **k)
        ev[1].record()
        torch.cuda.synchronize()
        return out, ev[0].elapsed_time(ev[1])

    for it in range(steps):
        row = {"step": it}
        oz, tz = timed(zero)
        row["zero"] = {"cycles": _cycles(oz["stats"]), "ms": tz}
        warm.set_config(start=mgfr.START_PREVIOUS if it > 0 else mgfr.START_ZERO)
        ow, tw = timed(warm)
        row["previous"] = {"cycles": _cycles(ow["stats"]), "ms": tw}
        diff = float(torch.abs(ow["fr"] / oz["fr"] - 1.0).max())
        oa, ta = timed(wall)
        row["previous_all"] = {"cycles": _cycles(oa["stats"]), "ms": ta}
        diff = max(diff, float(torch.abs(oa["fr"] / oz["fr"] - 1.0).max()))
        if lrn is not None:
            ol, tl = timed(lrn)
            row["learned"] = {"cycles": _cycles(ol["stats"]), "ms": tl}
            diff = max(diff, float(torch.abs(ol["fr"] / oz["fr"] - 1.0).max()))
        row["max_rel_diff_fr"] = diff
        acc, _ = warm.pm_accel(pos, 0, mgfr.PM_TOTAL)
        if kick is None:  # the toy's step size, fixed once
            amax = float(torch.abs(acc).max())
            n = max(steps, 1)
            kick = move_cells * (box / N_base) / (0.5 * n * (n + 1) * max(amax, 1e-300))
        mgfr.kick_drift(pos, vel, acc, kick, 1.0, box)
        rows.append(row)
    torch.cuda.synchronize()
    for s in (warm, zero, wall, lrn):
        if s is not None:
            s.close()
    return rows
