"""GPU parity of the particle-mesh potential (Sec. 2.4, Eq. (30)) against the
oracle: the density contrast assigned to PM grids of levels 0..2 (effective
mass, matter, both) to 1e-12, and the potential of the library's FP64 linear
multigrid (run to a 1e-12 relative residual) against the exact FFT solution
of the same 7-point problem to 1e-8 relative (the residual bound times the
condition number, about (N_pm / pi)^2 <= 420 here)."""
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


@pytest.mark.parametrize("prec,a", [(mgfr.PREC_FP64, 1.0), (mgfr.PREC_MIXED, 0.5)])
def test_pm_potential_matches_oracle(dev, prec, a):
    N0, box, fr0 = 16, 50.0, 1e-5
    d = synth.lognormal_delta(N0, box, 1.5, 13001)
    pos = synth.poisson_particles(d, box, 2.0, 13002)
    s = mgfr.Solver(0, fr0_abs=fr0, precision=prec, max_level=2)
    s.solve_particles(torch.from_numpy(pos).to(dev), N0, box, a)
    A = oracle.AMR(pos, N0, box, 2, 8)
    assert A.nlev == 3
    A.deposit()
    A.set_model(fr0, a=a)
    for l in range(A.nlev):  # the GPU's u in the oracle's cell order
        u = s.level_field(l, mgfr.FIELD_U)
        if l == 0:
            A.set_u(0, u)
        else:
            perm = np.argsort(s.level_keys(l), kind="stable")
            A.set_u(l, u[(8 * perm[:, None] + np.arange(8)[None, :]).ravel()])
    s.set_config(tol_rel=1e-12, max_vcycles=200)
    for lpm in (0, 1, 2):
        for what in (mgfr.PM_EFFECTIVE, mgfr.PM_MATTER, mgfr.PM_TOTAL):
            phi, dens, st = s.pm_potential(N0, lpm, what, want_density=True)
            want_d = A.density_pm(lpm, what)
            np.testing.assert_allclose(dens.cpu().numpy(), want_d, rtol=1e-12, atol=1e-12)
            want = A.pm_potential(lpm, what)
            got = phi.cpu().numpy()
            err = np.abs(got - want).max() / np.abs(want).max()
            assert err <= 1e-8, (lpm, what, err)
            assert abs(got.mean()) <= 1e-12 * np.abs(want).max()
            assert st["res_l2_final"] <= 1e-12 * st["f_l2"] and st["vcycles"] >= 1
    with pytest.raises(mgfr.MGFRError) as e:  # beyond 1024 cells per axis
        s.pm_potential(N0, 7, mgfr.PM_TOTAL)
    assert e.value.status == mgfr.MGFR_E_INVALID
    s.close()


def test_pm_potential_needs_a_particle_solve(dev):
    s = mgfr.Solver(0)
    phi = torch.empty((16,) * 3, dtype=torch.float64, device=dev)
    st = mgfr.lib().mgfr_pm_potential(s.h, 0, mgfr.PM_TOTAL, mgfr._ptr(phi), None, None)
    assert st == mgfr.MGFR_E_INVALID
    s.close()


def test_pm_accel_and_kick_drift_match_oracle(dev):
    """The PM force at the particles (Sec. 2.4, long-range part of Eq. (30))
    against the oracle's central differences and cloud-in-cell interpolation
    of its exact potential, and one leapfrog kick-drift step (exact FP64
    arithmetic on both sides: x + d (v + k a), wrapped)."""
    N0, box, fr0 = 16, 50.0, 1e-5
    d = synth.lognormal_delta(N0, box, 1.5, 13011)
    pos = synth.poisson_particles(d, box, 2.0, 13012)
    s = mgfr.Solver(0, fr0_abs=fr0, max_level=2, tol_rel=1e-12, max_vcycles=200)
    pt = torch.from_numpy(pos).to(dev)
    s.solve_particles(pt, N0, box)
    A = oracle.AMR(pos, N0, box, 2, 8)
    A.deposit()
    A.set_model(fr0)
    for l in range(A.nlev):
        u = s.level_field(l, mgfr.FIELD_U)
        if l == 0:
            A.set_u(0, u)
        else:
            perm = np.argsort(s.level_keys(l), kind="stable")
            A.set_u(l, u[(8 * perm[:, None] + np.arange(8)[None, :]).ravel()])
    for lpm, what in ((0, mgfr.PM_TOTAL), (1, mgfr.PM_MATTER), (2, mgfr.PM_EFFECTIVE)):
        acc, st = s.pm_accel(pt, lpm, what)
        want = oracle.pm_accel(A.pm_potential(lpm, what), box, pos)
        err = np.abs(acc.cpu().numpy() - want).max() / np.abs(want).max()
        assert err <= 1e-8, (lpm, what, err)
    vel = torch.zeros_like(pt)
    rng = np.random.default_rng(3)
    v0 = rng.standard_normal(pos.shape)
    vel.copy_(torch.from_numpy(v0))
    acc, _ = s.pm_accel(pt, 0, mgfr.PM_TOTAL)
    a_h = acc.cpu().numpy()
    p1 = pt.clone()
    mgfr.kick_drift(p1, vel, acc, 1e-3, 0.7, box)
    torch.cuda.synchronize()
    v1 = v0 + 1e-3 * a_h
    x1 = pos + 0.7 * v1
    x1 -= box * np.floor(x1 / box)
    np.testing.assert_array_equal(vel.cpu().numpy(), v1)
    np.testing.assert_array_equal(p1.cpu().numpy(), x1)
    s.close()
