"""GPU tests of the learned-start network: its BF16 tensor-core convolution
kernels against the FP64 NumPy oracle (forward, input gradient, weight
gradient), one whole training step and prediction against the network
oracle, and the trained network's gain over a zero start.

Tolerances: forward output is BF16, so |diff| <= 8e-3 max|ref|; the
gradients are accumulated and returned in FP32: |diff| <= 2e-5 max|ref|.
"""
import numpy as np
import pytest
import torch

from oracle import nn_oracle as nn
from paper_1305_2418_gb300 import build, learned, mgfr, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU test run without a GPU"
    build.build()
    return torch.device("cuda:0")


def bf(a, dev):
    return torch.from_numpy(a).to(dev).to(torch.bfloat16)


@pytest.mark.parametrize("B,D,Cin,Cout", [(1, 8, 16, 16), (2, 8, 48, 16), (1, 8, 192, 64),
                                          (1, 4, 64, 128), (1, 8, 96, 32), (2, 4, 128, 128),
                                          (2, 16, 32, 64), (4, 16, 16, 32),
                                          # the halo-tiled full-resolution kernels
                                          (1, 16, 16, 16), (2, 16, 48, 16), (1, 32, 16, 16),
                                          (1, 16, 16, 32), (2, 16, 32, 32), (1, 16, 32, 16),
                                          # the streamed-weight halo kernels
                                          (1, 16, 96, 32), (1, 16, 32, 64), (1, 16, 64, 64),
                                          (1, 16, 64, 128), (1, 16, 128, 128), (1, 16, 192, 64)])
def test_conv_kernels_match_oracle(dev, B, D, Cin, Cout):
    rng = np.random.default_rng(B * 1000 + D * 10 + Cin + Cout)
    x = rng.standard_normal((B, D, D, D, Cin)).astype(np.float32)
    W = (rng.standard_normal((27, Cin, Cout)) / np.sqrt(27 * Cin)).astype(np.float32)
    b = rng.standard_normal(Cout).astype(np.float32)
    g = rng.standard_normal((B, D, D, D, Cout)).astype(np.float32)
    xt, Wt, gt = bf(x, dev), bf(W, dev), bf(g, dev)
    # the oracle sees exactly the BF16-rounded operands, in FP64
    x64 = xt.float().cpu().numpy().astype(np.float64)
    W64 = Wt.float().cpu().numpy().astype(np.float64)
    g64 = gt.float().cpu().numpy().astype(np.float64)
    bt = torch.from_numpy(b).to(dev)
    y = mgfr.conv3d(0, xt, Wt, bias=bt, relu=True).float().cpu().numpy()
    y_ref = nn.conv3d_fwd(x64, W64, b.astype(np.float64), relu=True)
    assert np.abs(y - y_ref).max() <= 8e-3 * np.abs(y_ref).max()
    gx = mgfr.conv3d(1, xt, Wt, g=gt).cpu().numpy()
    gx_ref = nn.conv3d_dgrad(g64, W64)
    assert np.abs(gx - gx_ref).max() <= 2e-5 * np.abs(gx_ref).max()
    db = torch.empty(Cout, dtype=torch.float32, device=dev)
    dW = mgfr.conv3d(2, xt, Wt, g=gt, db=db).cpu().numpy()
    dW_ref, db_ref = nn.conv3d_wgrad(x64, g64)
    assert np.abs(dW - dW_ref).max() <= 2e-5 * np.abs(dW_ref).max()
    assert np.abs(db.cpu().numpy() - db_ref).max() <= 2e-5 * np.abs(db_ref).max()


def _rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def test_unet_training_step_matches_oracle(dev):
    """One training step of the whole network through the C ABI (features, 14
    convolutions, pooling, upsampling, concatenation, head, loss in v,
    backward pass, Adam) against the FP64 network oracle, which rounds to
    bfloat16 where the library stores bfloat16: the loss, every parameter
    block's gradient, the parameters after the Adam step, and the prediction.

    Tolerances.  The two sides differ by FP32 against FP64 accumulation in
    every layer, which moves some values across a bfloat16 rounding boundary
    (2^-8 relative), and those flips propagate.  The bound is calibrated on
    the oracle itself: its response (relative L2) to a 1e-7 relative change
    of the parameters, the size of an FP32 rounding, times 5, at least 5e-3.
    On this case that response is at most 0.8% for a gradient block and 0.3%
    for the prediction; a structural mistake (a swapped concatenation, a
    missing 1/8 in the pooling adjoint, a wrong tap) changes them by O(1).
    The loss must agree to 1e-3 and the Adam update, elementwise FP32 from the
    library's own gradient, to 1e-6 absolute."""
    D, box, fr0, lr = 32, 12.5, 1e-5, 1e-3
    s = mgfr.Solver(0, precision=mgfr.PREC_MIXED)
    s.unet_init(seed=21)
    P0 = s.unet_params()
    delta = synth.lognormal_delta(D, box, 1.5, 31)
    ut = 0.05 * synth.gaussian_field(D, box, 1.0, 32) - 0.5
    dd = torch.from_numpy(delta).to(dev)
    loss = s.unet_train_step(dd[None].contiguous(), np.array([fr0]),
                             torch.from_numpy(ut).to(dev)[None].contiguous(), lr=lr)
    G = s.unet_grads()
    P1 = s.unet_params()
    x0 = nn.features(delta, fr0)[None]

    def oracle_step(P):
        v, cache = nn.unet_forward(P, x0, bf16_storage=True)
        loss_, gv = nn.mse_v(v, ut[None])
        return loss_, nn.unet_backward(cache, gv, bf16_storage=True), v

    loss_ref, G_ref, _ = oracle_step(P0.astype(np.float64))
    rng = np.random.default_rng(5)
    Pp = P0.astype(np.float64) * (1.0 + 1e-7 * rng.standard_normal(P0.size))
    _, G_pert, _ = oracle_step(Pp)
    assert abs(loss / loss_ref - 1.0) <= 1e-3, (loss, loss_ref)
    offs, hoff, n = nn.param_layout()
    assert len(G) == n
    blocks = [(wo, bo) for (wo, bo), _ in zip(offs, nn.CONVS)]
    blocks += [(bo, bo + co) for (wo, bo), (_, co, _) in zip(offs, nn.CONVS)]
    blocks += [(hoff, n)]
    for lo, hi in blocks:
        tol = max(5.0 * _rel_l2(G_pert[lo:hi], G_ref[lo:hi]), 5e-3)
        err = _rel_l2(G[lo:hi], G_ref[lo:hi])
        assert err <= tol, (lo, hi, err, tol)
    P1_ref, _, _ = nn.adam_step(P0, G, np.zeros(n), np.zeros(n), 1, lr, dtype=np.float32)
    assert np.abs(P1 - P1_ref).max() <= 1e-6
    u = s.unet_predict(dd, fr0).cpu().numpy()
    v1, _ = nn.unet_forward(P1.astype(np.float64), x0, bf16_storage=True)
    v1p, _ = nn.unet_forward(P1.astype(np.float64) * (1.0 + 1e-7 * rng.standard_normal(n)), x0,
                             bf16_storage=True)
    u_ref = nn.U_SCALE * np.sinh(v1[0])
    tol = max(5.0 * _rel_l2(nn.U_SCALE * np.sinh(v1p[0]), u_ref), 5e-3)
    assert _rel_l2(u, u_ref) <= tol, (_rel_l2(u, u_ref), tol)
    s.close()


def test_unet_training_and_learned_start(dev):
    """Train on solver-generated 32^3 pairs (12.5 Mpc/h boxes: the 0.39 Mpc/h
    cell of the 256^3 / 100 Mpc/h fields), then start 64^3 solves at the same
    cell size from the prediction.  The polished answer must not depend on the
    start.  What the network must deliver: over the fields, a start closer to
    the solution (RMS in u, summed) than the zero start by a factor 2, at a
    cost of at most one more V-cycle per field.  It saves few V-cycles and no
    time to 1e-8 (measured and reported by bench.py): the first V-cycle from
    zero already brings the residual to a few per cent, and the prediction
    costs more than the cycles it saves."""
    s = mgfr.Solver(0, precision=mgfr.PREC_MIXED)
    deltas, fr0s, us = learned.make_training_set(s, 256, 32, 12.5, seed=11)
    s.unet_init(seed=3)
    # lr 1e-3: at 2e-3 the loss spikes (once to 94 times its first value) and
    # whether training recovers depends on the mini-batch seed and on FP32
    # summation order (two weight-gradient kernels that agree to 1e-6, seeds 5
    # and 6: two of the four runs ended above the bound below); at 1e-3 both
    # kernels reach 0.015-0.017 from 0.11-0.12
    losses = learned.train(s, deltas, fr0s, us, steps=2000, batch=4, lr=1e-3, seed=5)
    first, last = float(np.mean(losses[:20])), float(np.mean(losses[-20:]))
    # the output layer starts at zero, so the first losses are those of the
    # zero prediction; a quarter of them is half its RMS error in v, the same
    # factor the start error must reach below
    assert np.isfinite(last) and last < 0.25 * first, (first, last)
    rng = np.random.default_rng(99)
    fields = []
    for q in range(3):
        fr0 = [1e-6, 1e-5, 1e-4][q]
        d = torch.from_numpy(synth.lognormal_delta(64, 25.0, float(rng.uniform(0.5, 2.0)),
                                                   777 + q)).to(dev)
        fields.append((d, fr0))
    rows = learned.evaluate(s, fields, 25.0)
    for r in rows:
        # the polished answer does not depend on the start
        assert r["max_rel_diff_fr"] <= 1e-5, r
        assert np.isfinite(r["start_rms_err"]) and r["learned_cycles"] >= 1, r
        # a start costs at most one more V-cycle than zero
        assert r["learned_cycles"] <= r["zero_cycles"] + 1, r
    # the prediction is closer to the solution than zero
    err = sum(r["start_rms_err"] for r in rows)
    zero = sum(r["zero_rms_err"] for r in rows)
    assert err <= 0.5 * zero, (first, last, rows)
    s.close()
