"""Initial-guess modes of the solve calls (cfg.start) and the network's
parameter file, on a GPU: the user start needs u_init, the learned start
needs a network, a saved network loads back bit for bit, and a learned start
(dense, particle and batched solves) reaches the zero start's answer within
the mixed-precision tolerance (1e-5 relative on f_R)."""
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


def rel(a, b):
    return float(torch.abs(a / b - 1.0).max())


def test_start_modes_validate(dev):
    d = torch.from_numpy(synth.lognormal_delta(32, 50.0, 1.0, 12001)).to(dev)
    s = mgfr.Solver(0, precision=mgfr.PREC_MIXED, start=mgfr.START_USER)
    with pytest.raises(mgfr.MGFRError) as e:
        s.solve_density(d, 50.0)
    assert e.value.status == mgfr.MGFR_E_INVALID
    s.set_config(start=mgfr.START_LEARNED)  # no network yet
    with pytest.raises(mgfr.MGFRError) as e:
        s.solve_density(d, 50.0)
    assert e.value.status == mgfr.MGFR_E_INVALID
    s.unet_init(seed=4)
    with pytest.raises(mgfr.MGFRError) as e:  # the learned start takes no u_init
        s.solve_density(d, 50.0, u_init=torch.zeros_like(d))
    assert e.value.status == mgfr.MGFR_E_INVALID
    small = torch.from_numpy(synth.lognormal_delta(16, 50.0, 1.0, 12002)).to(dev)
    with pytest.raises(mgfr.MGFRError) as e:  # below the network's smallest box
        s.solve_density(small, 50.0)
    assert e.value.status == mgfr.MGFR_E_INVALID
    s.close()


def test_network_file_round_trip(dev, tmp_path):
    d = torch.from_numpy(synth.lognormal_delta(32, 12.5, 1.5, 12003)).to(dev)
    a = mgfr.Solver(0)
    a.unet_init(seed=7)
    path = str(tmp_path / "net.bin")
    a.unet_save(path)
    b = mgfr.Solver(0)
    b.unet_load(path)
    np.testing.assert_array_equal(a.unet_params(), b.unet_params())
    ua, ub = a.unet_predict(d, 1e-5), b.unet_predict(d, 1e-5)
    assert torch.equal(ua, ub)
    with open(path, "r+b") as fh:  # truncated file
        fh.truncate(1000)
    with pytest.raises(mgfr.MGFRError) as e:
        b.unet_load(path)
    assert e.value.status == mgfr.MGFR_E_INVALID
    a.close()
    b.close()


def test_learned_start_reaches_the_same_answer(dev):
    box = 25.0
    d = torch.from_numpy(synth.lognormal_delta(64, box, 1.5, 12004)).to(dev)
    z = mgfr.Solver(0, precision=mgfr.PREC_MIXED, fr0_abs=1e-5)
    ref = z.solve_density(d, box)
    s = mgfr.Solver(0, precision=mgfr.PREC_MIXED, fr0_abs=1e-5, start=mgfr.START_LEARNED)
    s.unet_init(seed=9)
    out = s.solve_density(d, box)
    assert rel(out["fr"], ref["fr"]) <= 1e-5
    assert out["stats"]["res_l2_final"] <= 1e-8 * out["stats"]["f_l2"]
    # and against the FP64 oracle directly (the mixed-form tolerance)
    u_ref, st_ref = oracle.solve_dense(d.cpu().numpy(), box, 1e-5, tol=1e-11, max_vcycles=300)
    assert st_ref["converged"] == 1.0
    fr_ref, _ = oracle.force_dense(u_ref, box, 1e-5)
    assert np.abs(out["fr"].cpu().numpy() / fr_ref - 1.0).max() <= 1e-5
    # particle solve: the base level is predicted from its deposited density
    N0, pbox = 32, 25.0
    pd = synth.lognormal_delta(N0, pbox, 1.5, 12005)
    pos = torch.from_numpy(synth.poisson_particles(pd, pbox, 1.0, 12006)).to(dev)
    for sv in (z, s):
        sv.set_config(max_level=1)
    pz = z.solve_particles(pos, N0, pbox)
    ps = s.solve_particles(pos, N0, pbox)
    assert rel(ps["fr"], pz["fr"]) <= 1e-5
    assert float(torch.abs(ps["acc"] - pz["acc"]).max() / torch.abs(pz["acc"]).max()) <= 1e-5
    # batch: items of 32^3 and more are predicted, the 16^3 one starts from zero
    sizes = [64, 16, 32, 32]
    deltas = [torch.from_numpy(synth.lognormal_delta(N, box, 1.2, 12010 + q)).to(dev)
              for q, N in enumerate(sizes)]
    fr0s = [1e-6, 1e-5, 1e-4, 3e-5]
    oz, stz = z.batch_solve(deltas, [box] * 4, fr0s)
    ol, stl = s.batch_solve(deltas, [box] * 4, fr0s)
    assert stz == mgfr.MGFR_OK and stl == mgfr.MGFR_OK
    for a_, b_ in zip(ol, oz):
        assert rel(a_["fr"], b_["fr"]) <= 1e-5
    z.close()
    s.close()
