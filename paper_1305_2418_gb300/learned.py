"""Learned initial guess: training data from the solver, training loop and
evaluation, on the library's own kernels (argument marshalling only).

The training pairs are (delta, u) with u the solution the batched solver
(mgfr_batch_solve) reaches at ||f - L(u)|| <= 1e-8 ||f||.  The network
(mgfr_unet_*) is fully convolutional; it is trained on small boxes and applied
to larger ones at the same cell size.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import mgfr, synth


def make_training_set(solver: "mgfr.Solver", n: int, D: int, box: float, seed: int,
                      sigma_range=(0.5, 2.0), fr0_range=(1e-6, 1e-4), chunk: int = 96):
    """n seeded lognormal fields of D^3 (sigma_g uniform, |fR0| log-uniform)
    and their solutions u, solved in batches of `chunk` in one launch each.
    Returns (deltas [n,D,D,D] CUDA FP64, fr0s (n,) numpy, u [n,D,D,D] CUDA FP64)."""
    import torch
    rng = np.random.default_rng(seed)
    dev = torch.device("cuda", solver.device)
    deltas = torch.empty((n, D, D, D), dtype=torch.float64, device=dev)
    us = torch.empty_like(deltas)
    fr0s = np.empty(n)
    for q in range(n):
        sig = rng.uniform(*sigma_range)
        fr0s[q] = 10 ** rng.uniform(math.log10(fr0_range[0]), math.log10(fr0_range[1]))
        deltas[q] = torch.from_numpy(synth.lognormal_delta(D, box, sig, seed * 100003 + q))
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        outs, _ = solver.batch_solve([deltas[q] for q in range(s, e)], [box] * (e - s),
                                     list(fr0s[s:e]), want_u=True)
        for q, o in zip(range(s, e), outs):
            us[q] = o["u"]
    return deltas, fr0s, us


def train(solver: "mgfr.Solver", deltas, fr0s, us, steps: int, batch: int = 4, lr: float = 1e-3,
          seed: int = 0, lr_final: float = 1e-4):
    """Adam steps on random mini-batches (cosine learning-rate decay).
    Returns the per-step losses."""
    rng = np.random.default_rng(seed)
    n = deltas.shape[0]
    losses = []
    for it in range(steps):
        idx = rng.choice(n, batch, replace=False)
        lr_t = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * it / max(steps, 1)))
        ti = __import__("torch").as_tensor(idx, device=deltas.device)
        losses.append(solver.unet_train_step(deltas.index_select(0, ti), fr0s[idx],
                                             us.index_select(0, ti), lr=lr_t))
    return losses


def solve_cycles(solver: "mgfr.Solver", delta, box: float, fr0: float, u_init=None):
    """Mixed-precision dense solve to 1e-8; returns (V-cycles incl. FP64 outer
    iterations, solve ms, stats)."""
    import torch
    solver.set_config(fr0_abs=fr0, precision=mgfr.PREC_MIXED)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = solver.solve_density(delta, box, 1.0, u_init=u_init, want_acc=False, want_u=True)
    torch.cuda.synchronize()
    ms = 1e3 * (time.perf_counter() - t0)
    st = out["stats"]
    return st["vcycles"] + st["outer_iters"], ms, out


def evaluate(solver: "mgfr.Solver", fields, box: float):
    """fields: list of (delta CUDA FP64, |fR0|).  For each, the V-cycles and
    time to 1e-8 from a zero start and from the network's prediction (the
    prediction time included)."""
    import torch
    rows = []
    for delta, fr0 in fields:
        z_cyc, z_ms, z_out = solve_cycles(solver, delta, box, fr0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u0 = solver.unet_predict(delta, fr0)
        torch.cuda.synchronize()
        p_ms = 1e3 * (time.perf_counter() - t0)
        l_cyc, l_ms, l_out = solve_cycles(solver, delta, box, fr0, u_init=u0)
        rel = float((torch.abs(l_out["fr"] / z_out["fr"] - 1.0)).max())
        rows.append({"fr0": fr0, "zero_cycles": z_cyc, "learned_cycles": l_cyc,
                     "zero_ms": z_ms, "learned_ms": l_ms + p_ms, "predict_ms": p_ms,
                     "start_rms_err": float(torch.sqrt(torch.mean((u0 - z_out["u"]) ** 2))),
                     "zero_rms_err": float(torch.sqrt(torch.mean(z_out["u"] ** 2))),
                     "max_rel_diff_fr": rel})
    return rows
