"""Parity of the particle path at the benchmark sizes, in the launch
configuration bench.py times (mixed precision, default configuration).

256^3 particles (the benchmarked workload): the whole hierarchy is compared
with the CPU oracle: sorted parent keys of every level bit-exact, counts
exact, leaf masses to 1e-12, and the oracle's own residual f - L(u) of the GPU
solution at sampled cells of every level (ghosts from the GPU's coarser
level) at the stopping level.

512^3 particles, 3 levels, |fR0| = 1e-6 (the largest workload): the same
comparison against the oracle's hierarchy, built at test time.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1305_2418_gb300 import build, mgfr, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU test run without a GPU"
    build.build()
    return torch.device("cuda:0")


def oct_cells(perm):
    return (8 * perm[:, None] + np.arange(8)[None, :]).ravel()


def test_particles256_against_oracle(dev):
    w = synth.WORKLOADS["particles256"]
    N, box, fr0, lmax = w["N"], w["box"], w["fr0"], w["lmax"]
    d = synth.lognormal_delta(N, box, w["sigma_g"], w["seed"])
    pos = synth.poisson_particles(d, box, w["nbar"], w["seed"])
    s = mgfr.Solver(0, precision=mgfr.PREC_MIXED, fr0_abs=fr0, max_level=lmax)
    out = s.solve_particles(torch.from_numpy(pos).to(dev), N, box)
    torch.cuda.synchronize()
    st = out["stats"]
    assert out["status"] == mgfr.MGFR_OK
    A = oracle.AMR(pos, N, box, lmax, 8)
    A.deposit()
    A.set_model(fr0)
    assert A.nlev == st["n_levels"] == lmax + 1
    rng = np.random.default_rng(7)
    perms = {}
    for l in range(A.nlev):
        if l == 0:
            cells = np.arange(A.ncell(0))
        else:
            keys = s.level_keys(l)
            perm = np.argsort(keys, kind="stable")
            np.testing.assert_array_equal(keys[perm], A.keys(l))
            cells = oct_cells(perm)
        perms[l] = cells
        np.testing.assert_array_equal(s.level_field(l, mgfr.FIELD_COUNT)[cells], A.counts(l))
        np.testing.assert_allclose(s.level_field(l, mgfr.FIELD_MASS)[cells], A.masses(l),
                                   rtol=1e-12, atol=1e-12)
        A.set_u(l, s.level_field(l, mgfr.FIELD_U)[cells])
    for l in range(A.nlev):
        f = A.source(l)
        sample = rng.choice(A.ncell(l), 3000, replace=False)
        r = A.residual_at(l, sample)
        # the level was stopped at ||r||_2 <= 1e-8 ||f||_2; pointwise the
        # residual stays far below the source scale
        assert np.abs(r).max() <= 1e-6 * np.abs(f).max(), (l, np.abs(r).max(), np.abs(f).max())
        assert st["level_res"][l] <= 1e-8 or l == 0
    assert st["res_l2_final"] <= 1e-8 * st["f_l2"]
    A.close()
    s.close()


def test_particles512_against_oracle(dev):
    """The 512^3 workload (3 levels, |fR0| = 1e-6) against the CPU oracle's
    hierarchy, built at test time (about 3 minutes on one core, 15 GB of host
    memory): sorted parent keys of every level bit-exact, counts exact, masses
    to 1e-12, and the oracle's residual of the GPU solution at sampled cells of
    every level, ghosts from the GPU's coarser level."""
    w = synth.WORKLOADS["particles512"]
    N, box, fr0, lmax = w["N"], w["box"], w["fr0"], w["lmax"]
    d = synth.lognormal_delta(N, box, w["sigma_g"], w["seed"])
    pos = synth.poisson_particles(d, box, w["nbar"], w["seed"])
    del d
    Np = pos.shape[0]
    s = mgfr.Solver(0, precision=mgfr.PREC_MIXED, fr0_abs=fr0, max_level=lmax)
    out = s.solve_particles(torch.from_numpy(pos).to(dev), N, box)
    torch.cuda.synchronize()
    st = out["stats"]
    assert out["status"] == mgfr.MGFR_OK
    assert st["n_levels"] == lmax + 1
    for l in range(1, st["n_levels"]):
        assert st["level_res"][l] <= 1e-8
    assert st["res_l2_final"] <= 1e-8 * st["f_l2"]
    A = oracle.AMR(pos, N, box, lmax, 8)
    assert A.nlev == st["n_levels"]
    A.deposit()
    A.set_model(fr0)
    rng = np.random.default_rng(11)
    total = 0.0
    for l in range(A.nlev):
        no, nc = s.level_info(l)
        assert nc == A.ncell(l)
        if l == 0:
            cells = np.arange(nc)
        else:
            keys = s.level_keys(l)
            perm = np.argsort(keys, kind="stable")
            np.testing.assert_array_equal(keys[perm], A.keys(l))
            del keys
            cells = oct_cells(perm)
            del perm
        np.testing.assert_array_equal(s.level_field(l, mgfr.FIELD_COUNT)[cells], A.counts(l))
        m_gpu = s.level_field(l, mgfr.FIELD_MASS)[cells]
        m_orc = A.masses(l)
        np.testing.assert_allclose(m_gpu, m_orc, rtol=1e-12, atol=1e-12)
        leaf = A.refined(l) == 0
        total += m_orc[leaf].sum()
        del m_gpu, m_orc, leaf
        A.set_u(l, s.level_field(l, mgfr.FIELD_U)[cells])
        del cells
    assert abs(total - Np) <= 1e-9 * Np  # leaf masses sum to the particle count
    for l in range(A.nlev):
        f = A.source(l)
        sample = rng.choice(A.ncell(l), 3000, replace=False)
        r = A.residual_at(l, sample)
        assert np.abs(r).max() <= 1e-6 * np.abs(f).max(), (l, np.abs(r).max(), np.abs(f).max())
        del f
    A.close()
    s.close()
