"""Time-stepped use on a GPU (Sec. 3.3, step 2): the previous step's
solution as the start (MGFR_START_PREVIOUS) in a toy particle-mesh loop.  The
answer must not depend on the start (1e-5 relative on the base f_R, the
mixed-precision tolerance), and once the particles have moved a little the
previous solution must cost fewer V-cycles than a zero start."""
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


def test_toy_pm_loop_previous_start(dev):
    N0, box = 32, 25.0
    d = synth.lognormal_delta(N0, box, 1.5, 14011)
    pos = torch.from_numpy(synth.poisson_particles(d, box, 2.0, 14012)).to(dev)
    rows = pmloop.run(pos, N0, box, steps=5, fr0=1e-5, max_level=2, move_cells=0.5)
    for r in rows:
        assert r["max_rel_diff_fr"] <= 1e-5, r
    prev = sum(r["previous"]["cycles"] for r in rows[1:])
    zero = sum(r["zero"]["cycles"] for r in rows[1:])
    assert prev < zero, rows
    assert torch.isfinite(pos).all() and float(pos.min()) >= 0.0 and float(pos.max()) < box
