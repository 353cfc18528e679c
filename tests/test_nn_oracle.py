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


def test_bf16_rounding_matches_torch():
    import torch
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.integers(-8, 8, 5000),
                        [0.0, 1.0, -1.0, 1.00390625, 1.01171875]])  # includes ties
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(nn.bf16(x), want)


def test_pool_and_upsample_explicit_loops():
    rng = np.random.default_rng(4)
    a = rng.standard_normal((2, 8, 8, 8, 3))
    p = nn.avgpool2(a)
    b, I, J, K, c = 1, 2, 0, 3, 2
    ref = sum(a[b, 2 * I + q, 2 * J + r, 2 * K + s, c] for q in (0, 1) for r in (0, 1)
              for s in (0, 1)) / 8.0
    assert np.isclose(p[b, I, J, K, c], ref, rtol=1e-14)
    up = nn.upsample2(p)
    for (i, j, k) in ((0, 0, 0), (5, 1, 6), (7, 7, 7)):
        assert up[b, i, j, k, c] == p[b, i // 2, j // 2, k // 2, c]


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(5)
    a = rng.standard_normal((1, 8, 8, 8, 2))
    c = rng.standard_normal((1, 4, 4, 4, 2))
    assert np.isclose((nn.avgpool2(a) * c).sum(), (a * nn.avgpool2_bwd(c)).sum(), rtol=1e-13)
    assert np.isclose((nn.upsample2(c) * a).sum(), (c * nn.upsample2_bwd(a)).sum(), rtol=1e-13)


def test_relu_and_mse_gradients_by_finite_differences():
    rng = np.random.default_rng(6)
    z = rng.standard_normal(200)
    z = z[np.abs(z) > 1e-3]
    R = rng.standard_normal(z.shape)
    g = nn.relu_bwd(R, np.maximum(z, 0.0))
    h = 1e-7
    fd = (np.maximum(z + h, 0) * R - np.maximum(z - h, 0) * R) / (2 * h)
    np.testing.assert_allclose(g, fd, atol=1e-7)
    out = rng.standard_normal(50)
    ut = 0.05 * rng.standard_normal(50)
    loss, gout = nn.mse_v(out, ut)
    for q in range(0, 50, 7):
        op, om = out.copy(), out.copy()
        op[q] += 1e-6
        om[q] -= 1e-6
        assert abs((nn.mse_v(op, ut)[0] - nn.mse_v(om, ut)[0]) / 2e-6 - gout[q]) < 1e-8
    # zero loss where the output is asinh(u / 0.01) exactly
    assert nn.mse_v(np.arcsinh(ut / 0.01), ut)[0] < 1e-28


def test_adam_closed_form():
    """From zero moments, and for a constant gradient, the bias-corrected
    moments are g and g^2, so each step moves p by -lr g / (|g| + eps)."""
    rng = np.random.default_rng(7)
    p0 = rng.standard_normal(40)
    g = rng.standard_normal(40)
    lr, eps = 1e-2, 1e-8
    p, m1, m2 = nn.adam_step(p0, g, np.zeros(40), np.zeros(40), 1, lr, eps=eps)
    np.testing.assert_allclose(p, p0 - lr * g / (np.abs(g) + eps), rtol=1e-13, atol=1e-15)
    p2, _, _ = nn.adam_step(p, g, m1, m2, 2, lr, eps=eps)
    np.testing.assert_allclose(p2, p0 - 2 * lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-15)


def test_features_screening_channel_is_the_uniform_solution():
    """Channel 3 is the solution for a uniform delta: with no gradients the
    oracle's periodic solve reduces to the local balance of Sec. 3.2."""
    import oracle
    for dval, fr0 in ((3.0, 1e-6), (0.5, 1e-5), (-0.4, 1e-5)):
        delta = np.full((8, 8, 8), dval)
        u, st = oracle.solve_dense(delta, 10.0, fr0, tol=1e-13, max_vcycles=200)
        x = nn.features(delta, fr0)
        want = np.arcsinh(u[0, 0, 0] / 0.01) / 5.0
        assert abs(x[0, 0, 0, 3] - want) < 1e-7 * max(1.0, abs(want))
        assert x[0, 0, 0, 0] == np.log(1.0 + dval)
        assert x[0, 0, 0, 1] == np.log10(fr0) + 5.0 and x[0, 0, 0, 2] == 1.0
        assert np.all(x[..., 4:] == 0.0)


def test_unet_gradient_by_finite_differences():
    """Whole-network parameter gradient (FP64, no bfloat16 rounding) against
    central differences of the loss, a few parameters in every block."""
    rng = np.random.default_rng(8)
    offs, hoff, n = nn.param_layout()
    P = 0.1 * rng.standard_normal(n)
    for (wo, bo), (ci, co, _) in zip(offs, nn.CONVS):  # He-normal scale
        P[wo:bo] *= 10.0 * np.sqrt(2.0 / (27 * ci))
    D = 8
    delta = np.exp(rng.standard_normal((D, D, D))) - 1.0
    x0 = nn.features(delta, 1e-5)[None]
    ut = 0.1 * rng.standard_normal((1, D, D, D))

    def loss(P_):
        v, _ = nn.unet_forward(P_, x0)
        return nn.mse_v(v, ut)[0]

    v, cache = nn.unet_forward(P, x0)
    _, gv = nn.mse_v(v, ut)
    G = nn.unet_backward(cache, gv)
    idx = [hoff + 3, hoff + 16]
    for (wo, bo), (ci, co, _) in zip(offs, nn.CONVS):
        idx += [wo + int(rng.integers(27 * ci * co)), bo + int(rng.integers(co))]
    h = 1e-6
    for q in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[q] += h
        Pm[q] -= h
        fd = (loss(Pp) - loss(Pm)) / (2 * h)
        assert abs(fd - G[q]) <= 1e-6 * max(1e-3, abs(fd)), (q, fd, G[q])
