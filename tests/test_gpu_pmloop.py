"""Time-stepped use on a GPU (Sec. 3.3, step 2): the previous step's
solution as the start in a toy particle-mesh loop, on the base level as the
paper's step list has it (MGFR_START_PREVIOUS) and on every level where the
octs persist (MGFR_START_PREVIOUS_ALL).  The answer must not depend on the
start (1e-5 relative on the base f_R, the mixed-precision tolerance); once
the particles have moved a little either previous solution must cost fewer
V-cycles than a zero start.  (Carrying it to the refined levels saves a few
more cycles than the base-level start alone on the 256^3-particle workload,
17.7 against 19.0 of 21 per step as bench.py measures, but not on this small
case, where the particles' motion changes the fine levels about as much as
the prolonged coarse solution misses them.)"""
import numpy as np
import pytest
import torch

from paper_1305_2418_gb300 import build, mgfr, pmloop, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU test run without a GPU"
    build.build()
    return torch.device("cuda:0")


def test_previous_start_validation(dev):
    N0, box = 32, 25.0
    d = synth.lognormal_delta(N0, box, 1.2, 14001)
    pos = torch.from_numpy(synth.poisson_particles(d, box, 1.0, 14002)).to(dev)
    s = mgfr.Solver(0, precision=mgfr.PREC_MIXED, start=mgfr.START_PREVIOUS, max_level=1)
    with pytest.raises(mgfr.MGFRError) as e:  # nothing solved yet
        s.solve_particles(pos, N0, box)
    assert e.value.status == mgfr.MGFR_E_INVALID
    s.set_config(start=mgfr.START_ZERO)
    s.solve_particles(pos, N0, box)
    s.set_config(start=mgfr.START_PREVIOUS)
    out = s.solve_particles(pos, N0, box)  # from its own converged solution
    assert out["stats"]["vcycles"] + out["stats"]["outer_iters"] <= 1
    with pytest.raises(mgfr.MGFRError) as e:  # another size
        s.solve_particles(pos, 16, box)
    assert e.value.status == mgfr.MGFR_E_INVALID
    s.close()


def test_previous_all_keys_and_first_solve(dev):
    """The start of the refined levels finds persisting octs by the Morton key
    of their parent cell, assuming the octs of every level are stored in
    increasing key order: checked here on the GPU's own keys.  On the first
    solve of a context nothing is held and the start is the zero start."""
    N0, box = 32, 25.0
    d = synth.lognormal_delta(N0, box, 1.5, 14021)
    pos = torch.from_numpy(synth.poisson_particles(d, box, 2.0, 14022)).to(dev)
    s = mgfr.Solver(0, precision=mgfr.PREC_MIXED, start=mgfr.START_PREVIOUS_ALL, max_level=3)
    z = mgfr.Solver(0, precision=mgfr.PREC_MIXED, max_level=3)
    o1 = s.solve_particles(pos, N0, box)
    oz = z.solve_particles(pos, N0, box)
    assert o1["stats"]["level_iters"] == oz["stats"]["level_iters"]
    for l in range(1, o1["stats"]["n_levels"]):
        keys = s.level_keys(l)  # parent linear index at level l - 1, storage order
        n = N0 << (l - 1)
        i, j, k = keys // (n * n), (keys // n) % n, keys % n
        m = np.zeros(keys.shape, dtype=np.uint64)
        for b in range(21):
            for v, sh in ((i, 2), (j, 1), (k, 0)):
                m |= ((v.astype(np.uint64) >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + sh)
        assert np.all(np.diff(m.astype(np.int64)) > 0), l
    # the same particles again: every oct persists, every level starts converged
    o2 = s.solve_particles(pos, N0, box)
    assert all(it <= 3 for it in o2["stats"]["level_iters"][1:o2["stats"]["n_levels"]]), o2["stats"]
    assert float(torch.abs(o2["fr"] / oz["fr"] - 1.0).max()) <= 1e-5
    s.close()
    z.close()


def test_toy_pm_loop_previous_start(dev):
    N0, box = 32, 25.0
    d = synth.lognormal_delta(N0, box, 1.5, 14011)
    pos = torch.from_numpy(synth.poisson_particles(d, box, 2.0, 14012)).to(dev)
    rows = pmloop.run(pos, N0, box, steps=5, fr0=1e-5, max_level=2, move_cells=0.5)
    for r in rows:
        assert r["max_rel_diff_fr"] <= 1e-5, r
    prev = sum(r["previous"]["cycles"] for r in rows[1:])
    prev_all = sum(r["previous_all"]["cycles"] for r in rows[1:])
    zero = sum(r["zero"]["cycles"] for r in rows[1:])
    assert prev < zero, rows
    assert prev_all < zero, rows
    assert torch.isfinite(pos).all() and float(pos.min()) >= 0.0 and float(pos.max()) < box
