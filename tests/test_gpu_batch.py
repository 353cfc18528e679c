"""Batched persistent solve (mgfr_batch_solve): many uneven periodic solves
in one cooperative launch, each at mixed-precision parity (<= 1e-5 relative
on f_R and force) with the CPU oracle; bounded grid-barrier waits; the
autotuner's choice."""
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


def make_batch(sizes, seed0, box=100.0):
    rng = np.random.default_rng(seed0)
    items = []
    for q, N in enumerate(sizes):
        sig = float(rng.uniform(0.5, 2.0))
        fr0 = float(10 ** rng.uniform(-6, -4))
        d = synth.lognormal_delta(N, box, sig, seed0 + q)
        items.append((N, d, fr0, box))
    return items


def test_batch_parity_with_oracle(dev):
    items = make_batch([8, 16, 32, 32, 16, 8, 32], 5000)
    s = mgfr.Solver(0, precision=mgfr.PREC_MIXED)
    deltas = [torch.from_numpy(d).to(dev) for (_, d, _, _) in items]
    outs, st = s.batch_solve(deltas, [b for (*_, b) in items], [f for (_, _, f, _) in items],
                             want_acc=True)
    torch.cuda.synchronize()
    assert st == mgfr.MGFR_OK
    for (N, d, fr0, box), o in zip(items, outs):
        u_ref, sr = oracle.solve_dense(d, box, fr0, tol=1e-11, max_vcycles=300)
        fr_ref, acc_ref = oracle.force_dense(u_ref, box, fr0)
        rel = np.abs(o["fr"].cpu().numpy() / fr_ref - 1.0).max()
        arel = np.abs(o["acc"].cpu().numpy() - acc_ref).max() / np.abs(acc_ref).max()
        assert rel <= 1e-5 and arel <= 1e-5, (N, fr0, rel, arel)
        assert o["stats"]["res_l2_final"] <= 1e-8 * o["stats"]["f_l2"]
    s.close()


def test_batch_mixed_sizes_against_oracle(dev):
    """Uneven sizes up to 128^3 in one launch: a 128^3, a 64^3 and a 32^3 item
    against the CPU oracle (f_R, force and u from the u output), the others
    against the single-solve FP64 path, whose oracle parity is tested
    elsewhere."""
    items = make_batch([128, 32, 64, 64, 32, 128, 64, 32], 6000)
    s = mgfr.Solver(0, precision=mgfr.PREC_MIXED)
    deltas = [torch.from_numpy(d).to(dev) for (_, d, _, _) in items]
    outs, st = s.batch_solve(deltas, [b for (*_, b) in items], [f for (_, _, f, _) in items],
                             want_acc=True, want_u=True)
    assert st == mgfr.MGFR_OK
    oracle.set_threads(0)
    try:
        for q, ((N, d, fr0, box), o, dd) in enumerate(zip(items, outs, deltas)):
            if q in (0, 1, 2):
                u_ref, sr = oracle.solve_dense(d, box, fr0, tol=1e-11, max_vcycles=300)
                assert sr["converged"] == 1.0
                fr_ref, acc_ref = oracle.force_dense(u_ref, box, fr0)
                assert np.abs(o["u"].cpu().numpy() - u_ref).max() <= 1e-5, (N, fr0)
            else:
                ref = mgfr.Solver(0, fr0_abs=fr0, tol_rel=1e-10)
                r = ref.solve_density(dd, box)
                fr_ref, acc_ref = r["fr"].cpu().numpy(), r["acc"].cpu().numpy()
                ref.close()
            rel = np.abs(o["fr"].cpu().numpy() / fr_ref - 1.0).max()
            arel = np.abs(o["acc"].cpu().numpy() - acc_ref).max() / np.abs(acc_ref).max()
            assert rel <= 1e-5 and arel <= 1e-5, (N, fr0, rel, arel)
    finally:
        oracle.set_threads(1)
    s.close()


def test_batch_scan_over_n_against_oracle(dev):
    """A parameter scan over the Hu-Sawicki exponent (n = 1, 2, 3; Sec. 2,
    Eq. (7)) and |fR0| through the batched path, each item against the
    oracle at its own n."""
    rng = np.random.default_rng(9100)
    cases = []
    for q, (N, n) in enumerate([(32, 1), (32, 2), (32, 3), (16, 2), (16, 3), (64, 2)]):
        fr0 = float(10 ** rng.uniform(-6, -4))
        d = synth.lognormal_delta(N, 100.0, float(rng.uniform(0.5, 2.0)), 9100 + q)
        cases.append((N, n, fr0, d))
    s = mgfr.Solver(0, precision=mgfr.PREC_MIXED)
    deltas = [torch.from_numpy(d).to(dev) for (*_, d) in cases]
    outs, st = s.batch_solve(deltas, [100.0] * len(cases), [f for (_, _, f, _) in cases],
                             ns=[n for (_, n, _, _) in cases], want_acc=True)
    assert st == mgfr.MGFR_OK
    oracle.set_threads(0)
    try:
        for (N, n, fr0, d), o in zip(cases, outs):
            u_ref, sr = oracle.solve_dense(d, 100.0, fr0, n=n, tol=1e-11, max_vcycles=300)
            assert sr["converged"] == 1.0
            fr_ref, acc_ref = oracle.force_dense(u_ref, 100.0, fr0, n=n)
            rel = np.abs(o["fr"].cpu().numpy() / fr_ref - 1.0).max()
            arel = np.abs(o["acc"].cpu().numpy() - acc_ref).max() / np.abs(acc_ref).max()
            assert rel <= 1e-5 and arel <= 1e-5, (N, n, fr0, rel, arel)
    finally:
        oracle.set_threads(1)
    s.close()


def test_batch_wait_limit_returns_timeout(dev):
    """A grid-barrier wait that runs out sets the error status and the kernel
    returns; the context stays usable."""
    items = make_batch([16, 16, 8], 7000)
    deltas = [torch.from_numpy(d).to(dev) for (_, d, _, _) in items]
    s = mgfr.Solver(0, precision=mgfr.PREC_MIXED, max_spins=0)
    with pytest.raises(mgfr.MGFRError) as ei:
        s.batch_solve(deltas, [100.0] * 3, [1e-5] * 3)
    assert ei.value.status == mgfr.MGFR_E_TIMEOUT
    s.set_config(max_spins=1 << 24)
    outs, st = s.batch_solve(deltas, [100.0] * 3, [1e-5] * 3)
    assert st == mgfr.MGFR_OK
    s.close()


def test_batch_autotune_and_warm_start(dev):
    items = make_batch([32, 16, 32], 8000)
    deltas = [torch.from_numpy(d).to(dev) for (_, d, _, _) in items]
    s = mgfr.Solver(0, precision=mgfr.PREC_MIXED)
    t, b = s.batch_autotune(deltas, [100.0] * 3, [f for (_, _, f, _) in items])
    assert t in (128, 256, 512) and b in (1, 2, 4)
    outs, st = s.batch_solve(deltas, [100.0] * 3, [f for (_, _, f, _) in items])
    assert st == mgfr.MGFR_OK
    # warm start from the solution: converged before any cycle
    u0 = [torch.log(o["fr"] / oracle.model_constants(f)["fbar"]) for o, (_, _, f, _) in
          zip(outs, items)]
    outs2, st2 = s.batch_solve(deltas, [100.0] * 3, [f for (_, _, f, _) in items], u_inits=u0)
    assert st2 == mgfr.MGFR_OK
    for o in outs2:
        assert o["stats"]["vcycles"] + o["stats"]["outer_iters"] <= 1
    s.close()
