"""The allocation-free entry point (mgfr_solve_density_noalloc) against the
context-based solve, through the C ABI, on a GPU.

Callers that cannot allocate device memory use the fixed in-library scratch;
its results must match mgfr_solve_density's FP64 path within the parity
tolerance (1e-6 relative on f_R and force), on calls in a row with
different inputs: two at the same size, so that the second finds the first
call's values in the same layout and must not use them, then a larger one.
This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1305_2418_gb300 import build, mgfr, synth

pytestmark = pytest.mark.gpu


def _noalloc(cfg, delta, box, a, stream):
    fr = torch.empty_like(delta)
    acc = torch.empty((3,) + tuple(delta.shape), dtype=delta.dtype, device=delta.device)
    st = mgfr.Stats()
    rc = mgfr.lib().mgfr_solve_density_noalloc(
        C.byref(cfg), C.c_void_p(delta.data_ptr()), delta.shape[0], box, a,
        C.c_void_p(fr.data_ptr()), C.c_void_p(acc.data_ptr()), C.c_void_p(stream.cuda_stream),
        C.byref(st))
    return rc, fr, acc, st


def test_noalloc_matches_context_solve_twice():
    assert torch.cuda.is_available(), "GPU test run without a GPU"
    build.build()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    box, fr0 = 100.0, 1e-5
    cfg = mgfr.default_config(fr0_abs=fr0)
    ref = mgfr.Solver(0, fr0_abs=fr0)
    # two calls at the same size with different fields (the second call's
    # scratch has the first call's layout and contents), then a larger size
    for seed, N, sig in ((11, 32, 1.0), (13, 32, 1.5), (12, 64, 1.5)):
        delta = torch.from_numpy(synth.lognormal_delta(N, box, sig, seed)).to(dev)
        rc, fr, acc, st = _noalloc(cfg, delta, box, 1.0, stream)
        torch.cuda.synchronize()
        assert rc == mgfr.MGFR_OK
        want = ref.solve_density(delta, box, 1.0)
        torch.cuda.synchronize()
        fr_r, acc_r = want["fr"].cpu().numpy(), want["acc"].cpu().numpy()
        assert np.abs(fr.cpu().numpy() / fr_r - 1.0).max() <= 1e-6
        assert np.abs(acc.cpu().numpy() - acc_r).max() <= 1e-6 * np.abs(acc_r).max()
        assert st.res_l2_final <= 1e-8 * st.f_l2
    ref.close()
    # sizes beyond the fixed scratch are rejected
    big = torch.zeros((128,) * 3, dtype=torch.float64, device=dev)
    rc, _, _, _ = _noalloc(cfg, big, box, 1.0, stream)
    assert rc == mgfr.MGFR_E_INVALID
