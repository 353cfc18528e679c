"""GPU parity of the particle path (mgfr_solve_particles) against the CPU
oracle: refinement structure bit-exact, deposited masses, per-level u and
f_R, and the force at the particles.

Tolerances: structure and counts exact; masses 1e-12 relative (FP64 atomics
change the summation order); FP64 path f_R per element and particle force
(max |diff| / max |ref|) <= 1e-6; mixed precision <= 1e-5.
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


def gpu_order_to_oracle(keys_gpu, keys_orc):
    """Row permutation taking GPU oct order to the oracle's (sorted) order."""
    perm = np.argsort(keys_gpu, kind="stable")
    np.testing.assert_array_equal(keys_gpu[perm], keys_orc)
    return perm


def run_case(dev, pos, N0, box, fr0, lmax, thr=8, prec=mgfr.PREC_FP64, a=1.0, tol_gpu=1e-8):
    s = mgfr.Solver(0, fr0_abs=fr0, precision=prec, max_level=lmax, refine_count=thr,
                    tol_rel=tol_gpu, max_vcycles=200)
    p = torch.from_numpy(np.ascontiguousarray(pos)).to(dev)
    out = s.solve_particles(p, N0, box, a)
    torch.cuda.synchronize()
    A = oracle.AMR(pos, N0, box, lmax, thr)
    A.deposit()
    A.set_model(fr0, a=a)
    rc, _ = A.solve(tol=1e-11, max_vcycles=300)
    assert rc == 0
    return s, out, A


def compare(s, out, A, N0, prec):
    tol = 1e-6 if prec == mgfr.PREC_FP64 else 1e-5
    nlev = out["stats"]["n_levels"]
    assert nlev == A.nlev
    for l in range(nlev):
        no, nc = s.level_info(l)
        assert nc == A.ncell(l)
        if l == 0:
            perm_cells = np.arange(nc)
        else:
            perm = gpu_order_to_oracle(s.level_keys(l), A.keys(l))
            perm_cells = (8 * perm[:, None] + np.arange(8)[None, :]).ravel()
        cnt = s.level_field(l, mgfr.FIELD_COUNT)[perm_cells]
        np.testing.assert_array_equal(cnt, A.counts(l))
        mass = s.level_field(l, mgfr.FIELD_MASS)[perm_cells]
        np.testing.assert_allclose(mass, A.masses(l), rtol=1e-12, atol=1e-12)
        fr_ref, acc_ref = A.level_force(l)
        fr = s.level_field(l, mgfr.FIELD_FR)[perm_cells]
        rel = np.abs(fr / fr_ref - 1.0).max()
        assert rel <= tol, (l, rel)
    acc_p = out["acc"].cpu().numpy()
    acc_ref = A.particle_force()
    arel = np.abs(acc_p - acc_ref).max() / np.abs(acc_ref).max()
    assert arel <= tol, arel
    return arel


@pytest.mark.parametrize("prec", [mgfr.PREC_FP64, mgfr.PREC_MIXED])
@pytest.mark.parametrize("N0,sig,fr0,lmax,nbar", [
    (32, 1.5, 1e-5, 2, 1.0),   # the 256^3-particle workload's parameters, small
    (32, 2.0, 1e-6, 3, 1.0),   # stiff, three refinement levels
    (16, 1.0, 1e-4, 1, 4.0),   # unscreened, denser sampling
])
def test_particle_parity(dev, prec, N0, sig, fr0, lmax, nbar):
    box = 100.0
    d = synth.lognormal_delta(N0, box, sig, 3000 + N0 + lmax)
    pos = synth.poisson_particles(d, box, nbar, 3100 + N0)
    s, out, A = run_case(dev, pos, N0, box, fr0, lmax, prec=prec)
    assert out["status"] == mgfr.MGFR_OK
    assert A.nlev > 1
    compare(s, out, A, N0, prec)
    s.close()


def test_full_refinement_equals_uniform_fine_solve(dev):
    """Refining every cell once: level 1 is a periodic (2N)^3 grid with no
    patch edge; it must equal the dense (2N)^3 solve of the same CIC delta."""
    N0, box, fr0 = 16, 50.0, 1e-5
    d = synth.lognormal_delta(2 * N0, box, 1.0, 50)
    pos = synth.poisson_particles(d, box, 2.0, 51)
    s = mgfr.Solver(0, fr0_abs=fr0, max_level=1, refine_count=-1, tol_rel=1e-10)
    s.solve_particles(torch.from_numpy(pos).to(dev), N0, box)
    B = oracle.AMR(pos, 2 * N0, box, 0, 8)
    B.deposit()
    dfine = B.delta(0).reshape((2 * N0,) * 3)
    uf, _ = oracle.solve_dense(dfine, box, fr0, tol=1e-11)
    keys = s.level_keys(1)
    u1 = s.level_field(1, mgfr.FIELD_U).reshape(-1, 2, 2, 2)
    pi, pj, pk = keys // (N0 * N0), (keys // N0) % N0, keys % N0
    dense = np.empty((2 * N0,) * 3)
    for a in (0, 1):
        for b in (0, 1):
            for c in (0, 1):
                dense[2 * pi + a, 2 * pj + b, 2 * pk + c] = u1[:, a, b, c]
    assert np.abs(dense - uf).max() < 1e-8
    s.close()


def test_edge_positions_and_tiny_inputs(dev):
    """Positions on and outside the box edges wrap periodically; a single
    particle and a single dense clump are valid inputs."""
    N0, box, fr0 = 16, 32.0, 1e-5
    rng = np.random.default_rng(2)
    edge = np.array([[0.0, 0.0, 0.0], [box, box / 2, 0.0], [-1e-9, 5.0, box - 1e-12],
                     [-box, 2 * box + 0.5, 3.0], [np.nextafter(box, 0), 1.0, 1.0]])
    clump = 7.0 + 0.3 * rng.random((200, 3))
    pos = np.concatenate([edge, clump, box * rng.random((300, 3))])
    s, out, A = run_case(dev, pos, N0, box, fr0, 3, prec=mgfr.PREC_FP64)
    assert A.nlev == 4
    compare(s, out, A, N0, mgfr.PREC_FP64)
    s.close()
    one = np.array([[3.3, 4.4, 5.5]])
    s, out, A = run_case(dev, one, 8, 10.0, fr0, 2, prec=mgfr.PREC_FP64)
    assert out["stats"]["n_levels"] == 1
    compare(s, out, A, 8, mgfr.PREC_FP64)
    s.close()


def test_invalid_particles_rejected(dev):
    s = mgfr.Solver(0, max_level=1)
    pos = torch.rand((100, 3), dtype=torch.float64, device=dev) * 10
    pos[7, 1] = float("nan")
    with pytest.raises(mgfr.MGFRError) as ei:
        s.solve_particles(pos, 16, 10.0)
    assert ei.value.status == mgfr.MGFR_E_INVALID
    with pytest.raises(mgfr.MGFRError):
        s.solve_particles(pos[:0], 16, 10.0)
    ok = s.solve_particles(torch.rand((100, 3), dtype=torch.float64, device=dev) * 10, 16, 10.0)
    assert ok["status"] == mgfr.MGFR_OK
    s.close()


@pytest.mark.parametrize("prec", [mgfr.PREC_FP64, mgfr.PREC_MIXED])
def test_host_buffer_solve_matches_device_solve(dev, prec):
    """mgfr_solve_particles_host (positions and forces in page-locked host
    memory, the gather in chunks with overlapped copies) gives the force of
    the device-buffer call (to rounding: the deposit's FP64 atomics add in
    any order, 1e-11 of the largest force), and the oracle's within
    tolerance; it also accepts pageable host memory and an Np that is not a
    multiple of the chunk count."""
    N0, box, fr0 = 32, 100.0, 1e-5
    d = synth.lognormal_delta(N0, box, 1.5, 3041)
    pos = synth.poisson_particles(d, box, 1.0, 3141)[:-5]
    s = mgfr.Solver(0, fr0_abs=fr0, precision=prec, max_level=2, tol_rel=1e-8, max_vcycles=200)
    ref = s.solve_particles(torch.from_numpy(pos).to(dev), N0, box)["acc"].cpu()
    host = torch.from_numpy(pos).pin_memory()
    out = s.solve_particles_host(host, N0, box)
    assert out["acc"].is_pinned()
    same = lambda x: (x - ref).abs().max().item() <= 1e-11 * ref.abs().max().item()
    assert same(out["acc"])
    pageable = s.solve_particles_host(torch.from_numpy(pos.copy()), N0, box)
    assert same(pageable["acc"])
    A = oracle.AMR(pos, N0, box, 2, 8)
    A.deposit()
    A.set_model(fr0)
    rc, _ = A.solve(tol=1e-11, max_vcycles=300)
    assert rc == 0
    acc_ref = A.particle_force()
    tol = 1e-6 if prec == mgfr.PREC_FP64 else 1e-5
    assert np.abs(out["acc"].numpy() - acc_ref).max() / np.abs(acc_ref).max() <= tol
    with pytest.raises(mgfr.MGFRError) as ei:
        s.solve_particles_host(host, 12, box)  # base size not a power of two
    assert ei.value.status == mgfr.MGFR_E_INVALID
    s.close()
