"""Pins of the FP64 NumPy network primitives (oracle/nn_oracle.py): a
brute-force single-voxel convolution and central finite differences of the
forward map for both gradients.  CPU only."""
import numpy as np

from oracle import nn_oracle as nn


def test_conv_fwd_matches_explicit_sum():
    rng = np.random.default_rng(0)
    D, Cin, Cout = 4, 3, 2
    x = rng.standard_normal((2, D, D, D, Cin))
    W = rng.standard_normal((27, Cin, Cout))
    y = nn.conv3d_fwd(x, W)
    b, i, j, k = 1, 0, 3, 2
    ref = np.zeros(Cout)
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                tap = (dx + 1) * 9 + (dy + 1) * 3 + (dz + 1)
                ref += x[b, (i + dx) % D, (j + dy) % D, (k + dz) % D] @ W[tap]
    assert np.allclose(y[b, i, j, k], ref, rtol=1e-13, atol=1e-13)


def test_conv_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    D, Cin, Cout = 4, 2, 3
    x = rng.standard_normal((1, D, D, D, Cin))
    W = rng.standard_normal((27, Cin, Cout))
    R = rng.standard_normal((1, D, D, D, Cout))
    loss = lambda x_, W_: float((nn.conv3d_fwd(x_, W_) * R).sum())
    gx = nn.conv3d_dgrad(R, W)
    dW, db = nn.conv3d_wgrad(x, R)
    h = 1e-6
    for _ in range(12):
        idx = tuple(rng.integers(0, s) for s in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        assert abs((loss(xp, W) - loss(xm, W)) / (2 * h) - gx[idx]) < 1e-6
        widx = tuple(rng.integers(0, s) for s in W.shape)
        Wp, Wm = W.copy(), W.copy()
        Wp[widx] += h
        Wm[widx] -= h
        assert abs((loss(x, Wp) - loss(x, Wm)) / (2 * h) - dW[widx]) < 1e-6
    assert np.allclose(db, R.reshape(-1, Cout).sum(0))


def test_pool_and_upsample_are_adjoint_up_to_scale():
    rng = np.random.default_rng(2)
    a = rng.standard_normal((1, 8, 8, 8, 3))
    c = rng.standard_normal((1, 4, 4, 4, 3))
    # <pool(a), c> = <a, up(c)> / 8
    assert np.isclose((nn.avgpool2(a) * c).sum(), (a * nn.upsample2(c)).sum() / 8.0)
