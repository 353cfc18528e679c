"""GPU parity of the effective mass density (Sec. 2.4) against the oracle:
per level, from the GPU's own u and masses (the formula), and on PM grids of
levels 0..3 (the volume-overlap assignment), to 1e-12.  One case leaves
a = 1, n = 1 and Omega_m = 0.3, so that the a^-3 factor, the exponent and
the matter density of the conversion are exercised."""
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


@pytest.mark.parametrize("prec,a,n,om", [
    (mgfr.PREC_FP64, 1.0, 1, 0.3),
    (mgfr.PREC_MIXED, 1.0, 1, 0.3),
    (mgfr.PREC_FP64, 0.5, 2, 0.25),
])
def test_effective_density_matches_oracle(dev, prec, a, n, om):
    N0, box, fr0 = 16, 50.0, 1e-5
    d = synth.lognormal_delta(N0, box, 1.5, 4001)
    pos = synth.poisson_particles(d, box, 2.0, 4002)
    s = mgfr.Solver(0, fr0_abs=fr0, precision=prec, max_level=2, tol_rel=1e-8, n=n, omega_m=om)
    s.solve_particles(torch.from_numpy(pos).to(dev), N0, box, a)
    A = oracle.AMR(pos, N0, box, 2, 8)
    A.deposit()
    A.set_model(fr0, a=a, n=n, omega_m=om)
    nlev = A.nlev
    assert nlev == 3
    for l in range(nlev):
        u = s.level_field(l, mgfr.FIELD_U)
        mass = s.level_field(l, mgfr.FIELD_MASS)
        Nl = N0 << l
        delta = mass * Nl ** 3 / len(pos) - 1.0
        got = s.effective_density(l).cpu().numpy()
        want = oracle.effective_density(u, delta, fr0, a=a, n=n, omega_m=om)
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-13)
        # the oracle hierarchy takes the GPU's u (oct order -> sorted keys)
        if l == 0:
            A.set_u(0, u)
        else:
            perm = np.argsort(s.level_keys(l), kind="stable")
            cells = (8 * perm[:, None] + np.arange(8)[None, :]).ravel()
            A.set_u(l, u[cells])
    for lpm in range(4):
        got = s.effective_mass_pm(N0, lpm).cpu().numpy()
        np.testing.assert_allclose(got, A.effective_pm(lpm), rtol=1e-12, atol=1e-12)
    s.close()


def test_level_getters_refuse_after_dense_solve(dev):
    """A dense solve reuses the workspace that holds a particle solve's base
    level: afterwards the level getters and the effective-density calls
    return MGFR_E_INVALID instead of reading stale or smaller arrays."""
    N0, box = 32, 50.0
    d = synth.lognormal_delta(N0, box, 1.5, 4011)
    pos = synth.poisson_particles(d, box, 1.0, 4012)
    s = mgfr.Solver(0, fr0_abs=1e-5, max_level=1)
    s.solve_particles(torch.from_numpy(pos).to(dev), N0, box)
    assert s.level_info(1)[0] > 0
    s.solve_density(torch.from_numpy(synth.lognormal_delta(16, box, 1.0, 4013)).to(dev), box)
    torch.cuda.synchronize()
    for call in (lambda: s.level_info(0), lambda: s.level_field(0, mgfr.FIELD_U),
                 lambda: s.effective_density(0), lambda: s.effective_mass_pm(N0, 0)):
        with pytest.raises(mgfr.MGFRError) as e:
            call()
        assert e.value.status == mgfr.MGFR_E_INVALID
    out = torch.empty(N0 ** 3, dtype=torch.float64, device=dev)
    assert mgfr.lib().mgfr_get_effective_density(s.h, 0, mgfr._ptr(out)) == mgfr.MGFR_E_INVALID
    assert mgfr.lib().mgfr_effective_mass_pm(s.h, 0, mgfr._ptr(out)) == mgfr.MGFR_E_INVALID
    # a new particle solve makes them valid again
    s.solve_particles(torch.from_numpy(pos).to(dev), N0, box)
    assert s.level_info(0)[1] == N0 ** 3
    s.close()
