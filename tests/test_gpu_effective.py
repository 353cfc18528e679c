"""GPU parity of the effective mass density (Sec. 2.4) against the oracle:
per level, from the GPU's own u and masses (the formula), and on PM grids of
levels 0..3 (the volume-overlap assignment), to 1e-12."""
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


@pytest.mark.parametrize("prec", [mgfr.PREC_FP64, mgfr.PREC_MIXED])
def test_effective_density_matches_oracle(dev, prec):
    N0, box, fr0 = 16, 50.0, 1e-5
    d = synth.lognormal_delta(N0, box, 1.5, 4001)
    pos = synth.poisson_particles(d, box, 2.0, 4002)
    s = mgfr.Solver(0, fr0_abs=fr0, precision=prec, max_level=2, tol_rel=1e-8)
    s.solve_particles(torch.from_numpy(pos).to(dev), N0, box)
    A = oracle.AMR(pos, N0, box, 2, 8)
    A.deposit()
    A.set_model(fr0)
    nlev = A.nlev
    assert nlev == 3
    for l in range(nlev):
        u = s.level_field(l, mgfr.FIELD_U)
        mass = s.level_field(l, mgfr.FIELD_MASS)
        Nl = N0 << l
        delta = mass * Nl ** 3 / len(pos) - 1.0
        got = s.effective_density(l).cpu().numpy()
        want = oracle.effective_density(u, delta, fr0)
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
