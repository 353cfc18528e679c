"""Parity of the particle path at the benchmark sizes, in the launch
configuration bench.py times (mixed precision, default configuration).

256^3 particles (the benchmarked workload): the whole hierarchy is compared
with the CPU oracle: sorted parent keys of every level bit-exact, counts
exact, leaf masses to 1e-12, and the oracle's own residual f - L(u) of the GPU
solution at sampled cells of every level (ghosts from the GPU's coarser
level) at the stopping level.

512^3 particles, 3 levels, |fR0| = 1e-6: the oracle's hierarchy build does not
finish in test time at this size, so properties that hold at any size are
checked: level-1 parent keys bit-exact against a dense NumPy brute force,
counts exact at sampled cells, mass conservation, the refinement rule, and
the oracle's residual of the base level at sampled cells.
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


def test_particles512_properties(dev):
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
    # base counts and level-1 keys by dense brute force (same FP64 expression)
    t = pos * (N / box)
    idx = np.floor(t).astype(np.int64) % N
    lin = (idx[:, 0] * N + idx[:, 1]) * N + idx[:, 2]
    cnt = np.bincount(lin, minlength=N ** 3)
    np.testing.assert_array_equal(s.level_field(0, mgfr.FIELD_COUNT).astype(np.int64), cnt)
    flag = (cnt > 8).reshape((N,) * 3)
    dil = np.zeros_like(flag)
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            for c in (-1, 0, 1):
                dil |= np.roll(flag, (a, b, c), axis=(0, 1, 2))
    keys1 = s.level_keys(1)
    np.testing.assert_array_equal(np.sort(keys1), np.flatnonzero(dil.ravel()))
    # refinement rule on every refined level: a refined cell exists; every
    # cell with more than 8 particles below the deepest level is refined
    for l in range(1, st["n_levels"] - 1):
        cl = s.level_field(l, mgfr.FIELD_COUNT)
        kids = s.level_keys(l + 1)
        no, _ = s.level_info(l)
        keys = s.level_keys(l)
        Nl = N << (l - 1)
        pi, pj, pk = keys // (Nl * Nl), (keys // Nl) % Nl, keys % Nl
        lin_l = np.empty(8 * no, dtype=np.int64)
        for ch in range(8):
            I, J, K = 2 * pi + (ch >> 2 & 1), 2 * pj + (ch >> 1 & 1), 2 * pk + (ch & 1)
            lin_l[ch::8] = (I * (2 * Nl) + J) * (2 * Nl) + K
        refined = np.isin(lin_l, kids)
        assert np.all(refined[cl > 8])
        assert np.isin(kids, lin_l).all()
    # mass conservation (leaf masses sum to the particle count)
    total = 0.0
    for l in range(st["n_levels"]):
        m = s.level_field(l, mgfr.FIELD_MASS)
        if l + 1 < st["n_levels"]:
            if l == 0:
                leaf = ~dil.ravel()
            else:
                no, _ = s.level_info(l)
                keys = s.level_keys(l)
                Nl = N << (l - 1)
                pi, pj, pk = keys // (Nl * Nl), (keys // Nl) % Nl, keys % Nl
                lin_l = np.empty(8 * no, dtype=np.int64)
                for ch in range(8):
                    I, J, K = 2 * pi + (ch >> 2 & 1), 2 * pj + (ch >> 1 & 1), 2 * pk + (ch & 1)
                    lin_l[ch::8] = (I * (2 * Nl) + J) * (2 * Nl) + K
                leaf = ~np.isin(lin_l, s.level_keys(l + 1))
            total += m[leaf].sum()
        else:
            total += m.sum()
    assert abs(total - Np) <= 1e-9 * Np
    assert abs(s.level_field(0, mgfr.FIELD_MASS).sum() - Np) <= 1e-9 * Np
    # the oracle's residual of the base level at sampled cells
    u0 = s.level_field(0, mgfr.FIELD_U)
    delta0 = s.level_field(0, mgfr.FIELD_MASS) * (N ** 3 / Np) - 1.0
    rng = np.random.default_rng(3)
    cells = rng.choice(N ** 3, 4000, replace=False)
    r = oracle.residual_dense_at(u0.reshape((N,) * 3), delta0.reshape((N,) * 3), cells, box, fr0)
    f = oracle.model_constants(fr0)["src"] * delta0
    assert np.abs(r).max() <= 1e-6 * np.abs(f).max()
    s.close()
