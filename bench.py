#!/usr/bin/env python
"""Benchmark of the f(R) field solve on GB300.

One step = one full particle solve of the 512^3 workload: 512^3 particles
Poisson-sampled from a lognormal field (sigma_g 2), 512^3 base grid with 3
refinement levels, |fR0| = 1e-6 (strongly screened), every level solved to
||f - L(u)|| <= 1e-8 ||f|| from a zero start with the mixed-precision form
(FP32 smoothing, FP64-accurate residual and defect correction), and the force
gathered to every particle.  Positions are resident in HBM when the timed
region starts.  The plain FP64 solve of the same input is timed beside it
(time-to-tolerance), and the other workloads are reported as extra keys.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun): every rank solves its own replica of the workload (the
solves are independent, no collective on the data path); the timing is the
max over ranks and `value` counts the updates of all ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1305_2418_gb300 import synth  # noqa: E402  (input generator only)

METRIC = ("cell-updates/s & time-to-residual 1e-8 per f(R) solve "
          "(plain FP64 vs mixed+learned), HBM %")
UNIT = "cell-updates/s"

WORKLOAD = dict(synth.WORKLOADS["particles512"], name="particles512", refine_count=8)
W256 = dict(synth.WORKLOADS["particles256"], name="particles256", refine_count=8)

# Algorithmic bytes per cell of one launch (what the method must move), per
# profiled kernel family:
#  0 FP32 NGS half-sweep (dense base level): read u (4) + f of the active
#    colour (2) + write the active u (2)            = 8 B per cell of the level
#  1 FP32 linear GS half-sweep on J e = r (base level): read u32 (4) + e (4) +
#    r active (2) + write e active (2)              = 12 B per cell
#  2 FP64-accurate residual of the level being solved, in double-float on the
#    FP32 pipes: read u, E, f pairs (24) + write r32, u32, e32 (12)
#                                                    = 36 B per cell; bound by
#    FP32/ALU issue (~270 operations per cell), not by HBM
#  3 NGS half-sweep on the octs of the refined level being solved (FP32, e^u
#    recomputed from u): as family 0               = 8 B per cell
#  4 FP32 linear GS half-sweep on the octs of the refined level: as family 1
#                                                    = 12 B per cell
# The oct families also read the face-neighbour table (6 ints per oct, 3 B per
# cell) and ghost faces; those are overhead of the refined-level layout, not
# bytes the method needs, and are not counted.
ALG_BYTES = {0: 8.0, 1: 12.0, 2: 36.0, 3: 8.0, 4: 12.0}
TABLE_BYTES = {0: 0.0, 1: 0.0, 2: 0.0, 3: 3.0, 4: 3.0}
FAMILY_BOUND = {0: "hbm", 1: "hbm", 2: "alu", 3: "hbm", 4: "hbm"}
# DRAM bytes per cell (dram__bytes_read.sum + dram__bytes_write.sum over the
# launch's cells), from ncu on the half-density 256^3-base sample of the same
# workload (same cell size, sigma_g, levels and |fR0|); scaled to a full
# launch by its cells (family 3: 343.6 MB over the 24.8 M cells of a level-1
# launch of that sample, 12124 x 256 threads, one per oct).
TRAFFIC_PER_CELL = {3: 343.59e6 / (12124 * 256 * 8)}
KERNEL_NAMES = {0: "k_sweep32 (FP32 NGS half-sweep, base level)",
                1: "k_lin_sweep (FP32 linear GS half-sweep, base level)",
                2: "k_resid_df / k_oresid_df (FP64-accurate residual in double-float)",
                3: "k_oct_sweep32<false> (FP32 NGS half-sweep on the octs of the refined level)",
                4: "k_oct_sweep32<true> (FP32 linear GS half-sweep on the octs of the refined level)"}
# FP64 form: FP64 operations per NGS point update counted from the kernels
# (6 faces x (E sum, half, difference, FMA as 2, two running sums) = 42; L and
# dL/du 10; step, clamp, update 4) = 56, plus one rsqrt (n = 1), one division
# and one exponential, which the FP64 pipe also executes but are not counted.
FP64_FLOPS_PER_UPDATE = 56.0
FP64_KERNEL_NAMES = {0: "k_sweep (FP64 NGS half-sweep, base level)",
                     3: "k_osweep<double> (FP64 NGS half-sweep on the octs of the refined level)"}
# GB300 FP64: 1.25 TFLOP/s nominal (about 2 FP64 FMA per clock per SM at
# 2.07 GHz on 152 SMs); no measured figure is available on this machine.
FP64_PEAK_TFLOPS = 1.25


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample of the workload
# ---------------------------------------------------------------------------
SAMPLE_N = 32


def _sample_inputs():
    w = WORKLOAD
    box = w["box"] * SAMPLE_N / w["N"]
    d = synth.lognormal_delta(SAMPLE_N, box, w["sigma_g"], w["seed"])
    pos = synth.poisson_particles(d, box, w["nbar"], w["seed"])
    return pos, box


def _oracle_particle_sample(threads: int):
    """One full oracle solve of a bounded sample of the workload: a 32^3 base
    grid in a 6.25 Mpc/h box (the workload's cell size), particles drawn the
    same way (nbar 1, sigma_g 2), the same refinement rule and levels, |fR0|
    and tolerance.  Returns (nonlinear cell updates, seconds)."""
    import oracle
    w = WORKLOAD
    oracle.set_threads(threads)
    pos, box = _sample_inputs()
    t0 = time.perf_counter()
    A = oracle.AMR(pos, SAMPLE_N, box, w["lmax"], w["refine_count"])
    A.deposit()
    A.set_model(w["fr0"], a=w["a"])
    rc, st = A.solve(tol=1e-8)
    A.particle_force()
    dt = time.perf_counter() - t0
    upd = st[3] + sum(st[4 + 4 * (l - 1)] * A.ncell(l) for l in range(1, A.nlev))
    A.close()
    oracle.set_threads(1)
    return upd, dt


def host_cpu() -> dict:
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "model": model, "machine": platform.machine()}


WORKLOAD_DESC = ("particles512: 512^3 particles Poisson-sampled (nbar 1) from a 512^3 lognormal "
                 "delta (sigma_g 2.0, P(k)~k^-1.5), box 100 Mpc/h, 512^3 base grid + 3 refinement "
                 "levels (> 8 particles, 1-cell buffer), adaptive CIC, |fR0| 1e-6, n 1, a 1; every "
                 "level solved to 1e-8 from a zero start; force gathered to the particles")

SAMPLE_DESC = ("full FP64 oracle particle solve (structure, adaptive CIC, every level to 1e-8, "
               "particle force) of a 32^3-base sample: box 6.25 Mpc/h (same cell size), nbar 1, "
               "sigma_g 2.0, 3 refinement levels, |fR0| 1e-6")


def cpu_baseline_sample(max_seconds: float = 12.0) -> dict:
    """The CPU oracle (FP64) on a bounded sample of the workload, on all host
    cores (OpenMP over each red-black colour; bit-identical to one thread) and
    on one core."""
    nproc = os.cpu_count() or 1
    res = {}
    for threads in (nproc, 1):
        t0 = time.perf_counter()
        upd = dt = 0.0
        n = 0
        while n < 1 or (time.perf_counter() - t0 < max_seconds and n < 6):
            u, t = _oracle_particle_sample(threads)
            upd += u
            dt += t
            n += 1
        res[threads] = (upd / dt, n, dt)
    v, n, dt = res[nproc]
    v1, n1, dt1 = res[1]
    return {"value": v, "unit": UNIT, "cores": nproc, "kind": "oracle",
            "sample": f"{n} x {SAMPLE_DESC}, {dt:.1f} s on {nproc} threads",
            "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                              "sample": f"{n1} x the same sample, {dt1:.1f} s"},
            "host": host_cpu()}


def run_reference(args, rank: int) -> None:
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        _oracle_particle_sample(threads)
    upd = dt = 0.0
    for _ in range(args.steps):
        u, t = _oracle_particle_sample(threads)
        upd += u
        dt += t
    val = upd / dt
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC, "parallelism": f"replicas x{args.gpus}"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": "one " + SAMPLE_DESC + " per step (a bounded sample "
                                       "of the workload), OpenMP over each red-black colour",
                             "host": host_cpu()},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# extra workloads (reported beside the headline)
# ---------------------------------------------------------------------------
def grid32_extra(mgfr, torch, dev, local):
    """32^3 periodic grid (delta lognormal, sigma_g 1), |fR0| 1e-5, plain FP64:
    V-cycles, device time per V-cycle and cell-updates/s (L2-resident, so no
    HBM roofline applies)."""
    w = synth.WORKLOADS["grid32"]
    d = torch.from_numpy(synth.lognormal_delta(w["N"], w["box"], w["sigma_g"], w["seed"])).to(dev)
    s = mgfr.Solver(local, fr0_abs=w["fr0"], precision=mgfr.PREC_FP64)
    for _ in range(3):
        s.solve_density(d, w["box"], w["a"], want_acc=False)
    rows = []
    for _ in range(20):
        o = s.solve_density(d, w["box"], w["a"], want_acc=False)
        rows.append(o["stats"])
    s.close()
    t = statistics.median(r["t_solve_ms"] for r in rows)
    vc = rows[0]["vcycles"]
    upd = rows[0]["cell_updates"]
    return {"workload": "grid32: 32^3 lognormal delta (sigma_g 1), box 100, |fR0| 1e-5, "
                        "plain FP64 to 1e-8",
            "vcycles": vc, "solve_ms": t, "us_per_vcycle": 1e3 * t / vc,
            "cell_updates_per_s": upd / (t / 1e3)}


def particles256_extra(mgfr, torch, dev, local, steps=5):
    """256^3 particles, 2 levels, |fR0| 1e-5: mixed step time and FP64
    time-to-tolerance."""
    w = W256
    d = synth.lognormal_delta(w["N"], w["box"], w["sigma_g"], w["seed"])
    pos = torch.from_numpy(synth.poisson_particles(d, w["box"], w["nbar"], w["seed"])).to(dev)
    out = {}
    for prec, name, k in ((mgfr.PREC_MIXED, "mixed", steps), (mgfr.PREC_FP64, "fp64", 1)):
        s = mgfr.Solver(local, fr0_abs=w["fr0"], precision=prec, max_level=w["lmax"])
        s.solve_particles(pos, w["N"], w["box"], w["a"], want_fr=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        upd = 0
        e0.record()
        for _ in range(k):
            st = s.solve_particles(pos, w["N"], w["box"], w["a"], want_fr=False)["stats"]
            upd += st["cell_updates"]
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / k
        out[name] = {"ms_per_solve": ms, "nonlinear_cell_updates_per_s": upd / k / (ms / 1e3)}
        s.close()
    return {"workload": "particles256: 256^3 particles (sigma_g 1.5), 256^3 base + 2 levels, "
                        "|fR0| 1e-5, to 1e-8", **out}


def batched_extra(mgfr, torch, dev, local, net_path=None):
    """96 independent periodic solves of 32^3/64^3/128^3 (about 32 each),
    sigma_g uniform in [0.5, 2], |fR0| log-uniform in [1e-6, 1e-4], box 100:
    one persistent launch (mixed precision, autotuned launch shape) against a
    sequential loop of plain FP64 solves on the same GPU; with a network, the
    same batch started from its predictions (the items of 32^3 and more,
    predicted per size before the launch)."""
    rng = np.random.default_rng(5000)
    sizes = [int(rng.choice([32, 64, 128])) for _ in range(96)]
    deltas, fr0s = [], []
    for q, N in enumerate(sizes):
        deltas.append(torch.from_numpy(synth.lognormal_delta(N, 100.0, float(rng.uniform(0.5, 2.0)),
                                                             5000 + q)).to(dev))
        fr0s.append(float(10 ** rng.uniform(-6, -4)))
    sb = mgfr.Solver(local, precision=mgfr.PREC_MIXED)
    t_shape = sb.batch_autotune(deltas, [100.0] * 96, fr0s)
    sb.batch_solve(deltas, [100.0] * 96, fr0s)
    torch.cuda.synchronize()
    reps = 3
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        outs, st = sb.batch_solve(deltas, [100.0] * 96, fr0s)
    e1.record()
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / reps
    ok = all(o["stats"]["res_l2_final"] <= 1e-8 * o["stats"]["f_l2"] for o in outs)
    learned_row = None
    if net_path:
        sb.set_config(start=mgfr.START_LEARNED)
        sb.unet_load(net_path)
        sb.batch_solve(deltas, [100.0] * 96, fr0s)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            outs_l, st_l = sb.batch_solve(deltas, [100.0] * 96, fr0s)
        e1.record()
        torch.cuda.synchronize()
        t_l = e0.elapsed_time(e1) / reps
        diff = max(float(torch.abs(a_["fr"] / b_["fr"] - 1.0).max()) for a_, b_ in zip(outs_l, outs))
        learned_row = {"batched_ms": t_l, "batched_solves_per_s": 96 / (t_l / 1e3),
                       "all_converged": all(o["stats"]["res_l2_final"] <= 1e-8 * o["stats"]["f_l2"]
                                            for o in outs_l),
                       "max_rel_diff_fr_vs_zero_start": diff,
                       "note": "network trained on 0.39 Mpc/h cells; these items have "
                               "0.78-3.1 Mpc/h cells"}
    s64 = mgfr.Solver(local, precision=mgfr.PREC_FP64)
    s64.solve_density(deltas[0], 100.0)
    torch.cuda.synchronize()
    e0.record()
    for d, f in zip(deltas, fr0s):
        s64.set_config(fr0_abs=f)
        s64.solve_density(d, 100.0, want_acc=False)
    e1.record()
    torch.cuda.synchronize()
    t_seq = e0.elapsed_time(e1)
    sb.close()
    s64.close()
    return {"workload": "96 periodic solves, N in {32,64,128} (%d/%d/%d), sigma_g U[0.5,2], "
                        "|fR0| log-uniform [1e-6,1e-4], box 100, to 1e-8" %
                        (sizes.count(32), sizes.count(64), sizes.count(128)),
            "batched_ms": t_batch, "batched_solves_per_s": 96 / (t_batch / 1e3),
            "sequential_fp64_ms": t_seq, "sequential_fp64_solves_per_s": 96 / (t_seq / 1e3),
            "speedup": t_seq / t_batch, "launch_shape": {"threads": t_shape[0],
                                                          "blocks_per_sm": t_shape[1]},
            "all_converged": ok, "learned_start": learned_row}


def learned_extra(mgfr, learned, torch, dev, local):
    """Learned start: the U-Net trained on 2000 solver-generated 64^3 samples
    (box 25, the 0.39 Mpc/h cell), then 256^3 / 100 Mpc/h fields, sigma_g in
    {0.5,1,1.5,2} x |fR0| in {1e-6,1e-5,1e-4}: V-cycles and time to 1e-8 from
    the prediction (prediction time included) against a zero start."""
    s = mgfr.Solver(local, precision=mgfr.PREC_MIXED)
    t0 = time.perf_counter()
    deltas, fr0s, us = learned.make_training_set(s, 2000, 64, 25.0, seed=4)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    s.unet_init(seed=1)
    steps, B = 1500, 4
    t0 = time.perf_counter()
    losses = learned.train(s, deltas, fr0s, us, steps=steps, batch=B, lr=1e-3, seed=2)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del deltas, us
    # conv FLOPs per training step (fwd + dgrad + wgrad = 3x the forward)
    convs = [(16, 16, 0), (16, 16, 0), (16, 32, 1), (32, 32, 1), (32, 64, 2), (64, 64, 2),
             (64, 128, 3), (128, 128, 3), (192, 64, 2), (64, 64, 2), (96, 32, 1), (32, 32, 1),
             (48, 16, 0), (16, 16, 0)]
    fwd = sum(2 * 27 * ci * co * (64 >> l) ** 3 for ci, co, l in convs) * B
    fields = []
    for q, sig in enumerate((0.5, 1.0, 1.5, 2.0)):
        for fr0 in (1e-6, 1e-5, 1e-4):
            d = torch.from_numpy(synth.lognormal_delta(256, 100.0, sig, 9000 + q)).to(dev)
            fields.append((d, fr0))
    rows = learned.evaluate(s, fields, 100.0)
    net_path = os.path.join(tempfile.mkdtemp(), "unet.bin")
    s.unet_save(net_path)  # for the time-stepped loop
    s.close()
    zc = [r["zero_cycles"] for r in rows]
    lc = [r["learned_cycles"] for r in rows]
    return {"training": {"samples": 2000, "D": 64, "steps": steps, "batch": B,
                         "data_gen_s": t_data, "train_s": t_train,
                         "loss_first": float(np.mean(losses[:20])),
                         "loss_last": float(np.mean(losses[-20:])),
                         "conv_tflops": 3 * fwd * steps / t_train / 1e12},
            "eval_256": {"zero_cycles_mean": float(np.mean(zc)),
                         "learned_cycles_mean": float(np.mean(lc)),
                         "zero_ms_mean": float(np.mean([r["zero_ms"] for r in rows])),
                         "learned_ms_mean": float(np.mean([r["learned_ms"] for r in rows])),
                         "predict_ms_mean": float(np.mean([r["predict_ms"] for r in rows])),
                         "start_rms_err_mean": float(np.mean([r["start_rms_err"] for r in rows])),
                         "zero_rms_err_mean": float(np.mean([r["zero_rms_err"] for r in rows])),
                         "max_rel_diff_fr": float(max(r["max_rel_diff_fr"] for r in rows)),
                         "fields": len(rows)},
            "net_path": net_path}


def time_stepped_extra(mgfr, torch, dev, local, net_path, steps=8):
    """The 256^3-particle workload moved through a toy particle-mesh loop
    (force of Eq. (30) on the base PM grid, leapfrog; the fastest particle
    moves about one base cell over the run): per step the V-cycles of all
    levels and the solve time from a zero start, from the previous step's
    solution on the base level (the paper's step list) and on every level
    where the octs persist, and from the learned start."""
    from paper_1305_2418_gb300 import pmloop
    w = W256
    d = synth.lognormal_delta(w["N"], w["box"], w["sigma_g"], w["seed"])
    pos = torch.from_numpy(synth.poisson_particles(d, w["box"], w["nbar"], w["seed"])).to(dev)
    rows = pmloop.run(pos, w["N"], w["box"], steps, w["fr0"], w["lmax"], net_path=net_path,
                      device=local)
    out = {"workload": "particles256 moved through %d toy PM steps (force of Eq. (30), "
                       "leapfrog, about one base cell in all)" % steps,
           "max_rel_diff_fr": max(r["max_rel_diff_fr"] for r in rows)}
    for k in ("zero", "previous", "previous_all", "learned"):
        if k in rows[0]:
            later = rows[1:]
            out[k] = {"cycles_mean": float(np.mean([r[k]["cycles"] for r in later])),
                      "ms_mean": float(np.mean([r[k]["ms"] for r in later]))}
    return out


def enhancement_extra(torch, dev, local):
    """The AMR-vs-fixed-grid test (Sec. 5.1) on a lognormal stand-in: 256^3
    particles (sigma_g 1.5) in a 100 Mpc/h box solved on a 64^3 fixed grid, a
    512^3 fixed grid and a 64^3 base with 3 refinement levels (peak 512^3);
    the ratio P(delta + delta_eff) / P(delta) on a 512^3 PM grid, and how far
    the AMR and 64^3 enhancements (ratio - 1) stray from the 512^3 one."""
    from paper_1305_2418_gb300 import enhance
    box = 100.0
    d = synth.lognormal_delta(256, box, 1.5, 5100)
    pos = torch.from_numpy(synth.poisson_particles(d, box, 1.0, 5100)).to(dev)
    out = {"workload": "256^3 particles (sigma_g 1.5), box 100 Mpc/h; fixed 64^3, fixed 512^3, "
                       "64^3 base + 3 levels; PM grid 512^3"}
    for fr0 in (1e-5, 1e-6):
        r = {}
        for name, N0, L in (("fixed64", 64, 0), ("fixed512", 512, 0), ("amr64_3", 64, 3)):
            k, ratio, _, _ = enhance.run(pos, box, fr0, N0, L, 512, device=local)
            r[name] = ratio
        e512 = r["fixed512"] - 1.0
        out[f"fr0_{fr0:g}"] = {
            "k": np.round(k, 4).tolist(),
            "ratio_fixed512": np.round(r["fixed512"], 5).tolist(),
            "ratio_amr64_3": np.round(r["amr64_3"], 5).tolist(),
            "ratio_fixed64": np.round(r["fixed64"], 5).tolist(),
            "amr_vs_fixed512_max_rel_dev_k_le_5": float(
                np.abs((r["amr64_3"] - 1.0) / e512 - 1.0)[k <= 5.0].max()),
            "fixed64_vs_fixed512_max_rel_dev_k_lt_0.5": float(
                np.abs((r["fixed64"] - 1.0) / e512 - 1.0)[k < 0.5].max())}
    return out


def family_table(kern_ms, kern_n, kern_cells, steps, peak):
    fams = []
    for q in range(5):
        if kern_n[q] == 0:
            continue
        a_ms = kern_ms[q] / kern_n[q]
        cells = kern_cells[q] / kern_n[q]
        gbs = ALG_BYTES[q] * cells / (a_ms / 1e3) / 1e9
        fams.append({"kernel": KERNEL_NAMES[q], "bound": FAMILY_BOUND[q],
                     "launches_per_step": kern_n[q] / steps, "avg_launch_us": 1e3 * a_ms,
                     "alg_bytes_per_cell": ALG_BYTES[q], "achieved_gbs": gbs,
                     "frac_of_hbm": gbs / peak,
                     "with_table_gbs": (ALG_BYTES[q] + TABLE_BYTES[q]) * cells / (a_ms / 1e3) / 1e9,
                     "ms_per_step": kern_ms[q] / steps})
    return fams


# Layers of the learned start's network for profiler captures of its
# convolution kernels: (fields, grid size, Cin, Cout, ops); op 0 forward, 1
# input gradient, 2 weight gradient.  16 -> 16 is the full-resolution layer
# (halo-tiled kernel), 64 -> 64 a third-level layer of a 256^3 field and
# 96 -> 32 the second level's concatenation (streamed-weight halo kernel),
# 192 -> 64 the third level's concatenation (per-tap kernel).
CONV_CASE = ((1, 128, 16, 16, (0, 1, 2)), (1, 64, 64, 64, (0, 1, 2)),
             (1, 128, 96, 32, (0,)), (1, 64, 192, 64, (0,)))


def conv_case(dev):
    """Every op of CONV_CASE once as a warm-up, once more (the launches to
    capture: the 8 matching `k_conv_|k_wgrad_tc` after the first 8), then 5
    timed repetitions of each op with CUDA events; one JSON line per op."""
    import torch
    from paper_1305_2418_gb300 import mgfr

    layers = []
    for i, (B, D, ci, co, ops) in enumerate(CONV_CASE):
        g = torch.Generator(device=dev).manual_seed(100 + i)
        x = (torch.randn((B, D, D, D, ci), device=dev, generator=g) * 0.5).to(torch.bfloat16)
        w = (torch.randn((27, ci, co), device=dev, generator=g) * 0.1).to(torch.bfloat16)
        gy = (torch.randn((B, D, D, D, co), device=dev, generator=g) * 0.5).to(torch.bfloat16)
        bias = torch.zeros(co, device=dev, dtype=torch.float32)
        db = torch.zeros(co, device=dev, dtype=torch.float32)
        for op in ops:
            if op == 0:
                f = (lambda x=x, w=w, b=bias: mgfr.conv3d(0, x, w, b, relu=True))
            elif op == 1:
                f = (lambda x=x, w=w, gy=gy: mgfr.conv3d(1, x, w, g=gy))
            else:
                f = (lambda x=x, w=w, gy=gy, db=db: mgfr.conv3d(2, x, w, g=gy, db=db))
            layers.append((B, D, ci, co, op, f))
    for _ in range(2):
        for *_, f in layers:
            f()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for B, D, ci, co, op, f in layers:
        e0.record()
        for _ in range(5):
            f()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 5
        flop = 2.0 * 27 * ci * co * B * D ** 3
        print(json.dumps({"fields": B, "D": D, "cin": ci, "cout": co,
                          "op": ("forward", "input_grad", "weight_grad")[op],
                          "ms": round(ms, 4), "tflops": round(flop / ms / 1e9, 1)}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other workloads (32^3 grid, 256^3 particles, batched, learned)")
    ap.add_argument("--only-mixed", action="store_true",
                    help="run only the timed mixed-precision steps (for profiler captures)")
    ap.add_argument("--profile-case", action="store_true",
                    help="a smaller sample of the workload for full-metric profiler captures: "
                         "256^3 base in a 50 Mpc/h box (same cell size), nbar 0.5")
    ap.add_argument("--conv-case", action="store_true",
                    help="only the network's convolution layers (for profiler captures of "
                         "the convolution kernels)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    args.warmup = max(args.warmup, 3)

    import torch
    import torch.distributed as dist
    from paper_1305_2418_gb300 import build, mgfr
    from paper_1305_2418_gb300 import dist as D

    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    if args.conv_case:
        conv_case(dev)
        return

    w = dict(WORKLOAD)
    if args.profile_case:
        w.update(N=256, box=50.0, nbar=0.5)
    delta_h = synth.lognormal_delta(w["N"], w["box"], w["sigma_g"], w["seed"])
    pos_h = synth.poisson_particles(delta_h, w["box"], w["nbar"], w["seed"])
    del delta_h
    pos = torch.from_numpy(pos_h).to(dev)
    n_part = pos_h.shape[0]

    def solver(prec, profile=1):
        return mgfr.Solver(local, fr0_abs=w["fr0"], precision=prec, profile=profile,
                           max_level=w["lmax"], refine_count=w["refine_count"])

    def step(s, want_fr=False):
        return s.solve_particles(pos, w["N"], w["box"], w["a"], want_fr=want_fr)

    if args.only_mixed:
        sm = solver(mgfr.PREC_MIXED, profile=0)
        for _ in range(args.warmup + args.steps):
            step(sm)
        torch.cuda.synchronize()
        sm.close()
        return

    # ---- plain FP64 solve: time to tolerance, FP64-pipe figures ----
    s64 = solver(mgfr.PREC_FP64)
    step(s64)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    o64 = step(s64)
    e1.record()
    torch.cuda.synchronize()
    t64 = e0.elapsed_time(e1)
    st64 = o64["stats"]
    s64.close()

    # ---- mixed-precision form: the timed steps (graphs replayed) ----
    sm = solver(mgfr.PREC_MIXED, profile=0)
    for _ in range(args.warmup):
        step(sm)
    torch.cuda.synchronize()
    barrier()
    clocks = Clocks(local)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    upd = lin = 0
    e0.record()
    for _ in range(args.steps):
        out = step(sm)
        st = out["stats"]
        launches += st["gpu_launches"]
        upd += st["cell_updates"]
        lin += st["linear_updates"]
    e1.record()
    torch.cuda.synchronize()
    barrier()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    value, ms_max = D.whole_job_rate(upd, ms, dev)
    lin_value, _ = D.whole_job_rate(lin, ms, dev)
    last = st

    # ---- end to end through the public API: host buffers, copies timed ----
    # (mgfr_solve_particles_host: positions copied in, the force copied back
    # chunk by chunk while it is gathered)
    host_in = torch.from_numpy(pos_h).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()

    def step_host():
        return sm.solve_particles_host(host_in, w["N"], w["box"], w["a"], acc_out=host_out)

    step_host()
    torch.cuda.synchronize()
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record()
    e2e_upd = 0
    for _ in range(args.steps):
        r = step_host()
        e2e_upd += r["stats"]["cell_updates"]
    f1.record()
    torch.cuda.synchronize()
    e2e_ms = f0.elapsed_time(f1)
    e2e_value, _ = D.whole_job_rate(e2e_upd, e2e_ms, dev)
    del host_in, host_out
    # ---- potential of matter + effective mass on the base PM grid (Eq. (30)) ----
    pm = {}
    for what, name in ((mgfr.PM_TOTAL, "total"), (mgfr.PM_EFFECTIVE, "effective")):
        sm.pm_potential(w["N"], 0, what)
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record()
        _, _, pst = sm.pm_potential(w["N"], 0, what)
        g1.record()
        torch.cuda.synchronize()
        pm[name] = {"ms": g0.elapsed_time(g1), "vcycles": pst["vcycles"],
                    "res_rel": pst["res_l2_final"] / pst["f_l2"],
                    "gs_cell_updates_per_s": pst["linear_updates"] / (g0.elapsed_time(g1) / 1e3)}
    pm["grid"] = f"{w['N']}^3 periodic PM grid (the base grid), FP64 linear multigrid to 1e-8"
    sm.close()

    # ---- the same steps with CUDA events around each profiled launch ----
    # (launched directly on the library's stream instead of from graphs)
    ksteps = min(args.steps, 5)
    kern_ms, kern_n, kern_cells = [0.0] * 6, [0] * 6, [0] * 6
    sp = solver(mgfr.PREC_MIXED, profile=1)
    step(sp)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record()
    for _ in range(ksteps):
        stp = step(sp)["stats"]
        for q in range(5):
            kern_ms[q] += stp["kern_ms"][q]
            kern_n[q] += stp["kern_launches"][q]
            kern_cells[q] += stp["kern_cells"][q]
    p1.record()
    torch.cuda.synchronize()
    ms_prof = p0.elapsed_time(p1)
    sp.close()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant profiled kernel family ----
    # (the double-float residual is bound by arithmetic issue, not by HBM, and
    # is reported in the family table only)
    peak, peak_kind = peaks()
    fam = max((q for q in range(5) if FAMILY_BOUND[q] == "hbm"), key=lambda q: kern_ms[q])
    avg_ms = kern_ms[fam] / max(kern_n[fam], 1)
    cells_per_launch = kern_cells[fam] / max(kern_n[fam], 1)
    bytes_per_launch = ALG_BYTES[fam] * cells_per_launch
    achieved = bytes_per_launch / (avg_ms / 1e3) / 1e9
    traffic = TRAFFIC_PER_CELL[fam] * cells_per_launch if fam in TRAFFIC_PER_CELL else None
    roof = {"bound": "hbm", "kernel": KERNEL_NAMES[fam], "achieved": achieved, "peak": peak,
            "peak_source": peak_kind, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "launches": kern_n[fam], "avg_launch_us": 1e3 * avg_ms,
            "cells_per_launch": cells_per_launch, "alg_bytes_per_cell": ALG_BYTES[fam],
            "alg_bytes_per_launch": bytes_per_launch,
            "kernel_share_of_step": kern_ms[fam] / ms_prof,
            "profiled_ms_per_step": ms_prof / ksteps,
            "families": family_table(kern_ms, kern_n, kern_cells, ksteps, peak)}
    fp64 = {"bound": "fp64", "peak_tflops": FP64_PEAK_TFLOPS, "peak_source": "nominal",
            "flops_per_update": FP64_FLOPS_PER_UPDATE, "families": []}
    for q in (0, 3):
        if st64["kern_launches"][q] == 0:
            continue
        a_ms = st64["kern_ms"][q] / st64["kern_launches"][q]
        cells = st64["kern_cells"][q] / st64["kern_launches"][q]
        tfl = FP64_FLOPS_PER_UPDATE * cells / 2 / (a_ms / 1e3) / 1e12  # half the cells update
        fp64["families"].append({"kernel": FP64_KERNEL_NAMES[q],
                                 "launches": st64["kern_launches"][q],
                                 "avg_launch_us": 1e3 * a_ms, "achieved_tflops": tfl,
                                 "frac": tfl / FP64_PEAK_TFLOPS,
                                 "ms_per_solve": st64["kern_ms"][q]})

    cpu = None if (args.no_cpu_baseline or world > 1) else cpu_baseline_sample()
    extras = {}
    if not args.no_extras:
        from paper_1305_2418_gb300 import learned
        extras["grid32"] = grid32_extra(mgfr, torch, dev, local)
        extras["particles256"] = particles256_extra(mgfr, torch, dev, local)
        extras["learned_start"] = learned_extra(mgfr, learned, torch, dev, local)
        net_path = extras["learned_start"].pop("net_path")
        extras["batched"] = batched_extra(mgfr, torch, dev, local, net_path)
        extras["time_stepped"] = time_stepped_extra(mgfr, torch, dev, local, net_path)
        extras["amr_vs_fixed"] = enhancement_extra(torch, dev, local)

    nl = last["n_levels"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+df64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC if not args.profile_case else
                   "profile sample of particles512: 256^3 base, box 50, nbar 0.5",
                   "particles": n_part,
                   "levels_cells": last["cells_per_level"][:nl],
                   "precision": "mixed (FP32 smoothing; residual and defect correction in "
                                "double-float, about 48-bit)",
                   "l2": "inputs larger than L2 (positions 3.2 GB; every level's arrays "
                         "above 129 MB but level 3's FP32 ones)",
                   "parallelism": f"replicas x{world}"},
        "value_counts": "nonlinear NGS cell updates (all levels) per second of the whole step",
        "linear_cell_updates_per_s": lin_value,
        "time_to_tol_ms": {"mixed": ms_max / args.steps, "fp64": t64},
        "vcycles": {"mixed_fp32": last["vcycles"], "mixed_outer_fp64": last["outer_iters"],
                    "fp64": st64["vcycles"],
                    "refined_levels_mixed": last["level_iters"][1:nl],
                    "refined_levels_fp64": st64["level_iters"][1:st64["n_levels"]]},
        "cell_updates_per_step": {"nonlinear": last["cell_updates"],
                                  "linear": last["linear_updates"],
                                  "fp64_path": st64["cell_updates"]},
        "res_rel_final": last["res_l2_final"] / last["f_l2"],
        "level_res": last["level_res"][:nl],
        "roofline": roof,
        "fp64_roofline": fp64,
        "clocks": ck,
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 24 * n_part,
                "d2h_bytes_per_step": 24 * n_part, "ms_per_step": e2e_ms / args.steps},
        "cpu_baseline": cpu,
        "pm_potential": pm,
        **extras,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
