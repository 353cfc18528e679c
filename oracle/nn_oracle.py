"""FP64 NumPy reference for the learned-start network's primitives.

TEST INFRASTRUCTURE ONLY.  Direct 3^3 convolutions with circular padding on
NDHWC arrays, written as a sum over the 27 taps of shifted copies (tap =
(dx+1)*9 + (dy+1)*3 + (dz+1) reads the input at offset (dx, dy, dz)), their
gradients, 2^3 average pooling and nearest upsampling.  The gradients are
pinned against central finite differences in tests/test_nn_oracle.py.
"""
import numpy as np


def _taps():
    for tap in range(27):
        yield tap, tap // 9 - 1, (tap // 3) % 3 - 1, tap % 3 - 1


def _shift(x, dx, dy, dz):
    """s[b, i, j, k] = x[b, i+dx, j+dy, k+dz] (periodic)."""
    return np.roll(x, shift=(-dx, -dy, -dz), axis=(1, 2, 3))


def conv3d_fwd(x, W, b=None, relu=False):
    """y[m, co] = sum_tap sum_ci x[m + d_tap, ci] W[tap, ci, co] (+ b) (ReLU)."""
    y = np.zeros(x.shape[:-1] + (W.shape[2],))
    for tap, dx, dy, dz in _taps():
        y += _shift(x, dx, dy, dz) @ W[tap]
    if b is not None:
        y += b
    if relu:
        y = np.maximum(y, 0.0)
    return y


def conv3d_dgrad(g, W):
    """Gradient w.r.t. the input of conv3d_fwd (no bias/ReLU) for output gradient g."""
    gx = np.zeros(g.shape[:-1] + (W.shape[1],))
    for tap, dx, dy, dz in _taps():
        gx += _shift(g, -dx, -dy, -dz) @ W[tap].T
    return gx


def conv3d_wgrad(x, g):
    """Gradients w.r.t. W [27, Cin, Cout] and the bias for output gradient g."""
    Cin, Cout = x.shape[-1], g.shape[-1]
    dW = np.zeros((27, Cin, Cout))
    gf = g.reshape(-1, Cout)
    for tap, dx, dy, dz in _taps():
        dW[tap] = _shift(x, dx, dy, dz).reshape(-1, Cin).T @ gf
    return dW, gf.sum(0)


def avgpool2(x):
    B, D = x.shape[0], x.shape[1]
    return x.reshape(B, D // 2, 2, D // 2, 2, D // 2, 2, -1).mean(axis=(2, 4, 6))


def upsample2(x):
    return x.repeat(2, axis=1).repeat(2, axis=2).repeat(2, axis=3)
