"""FP64 NumPy reference for the learned-start network.

TEST INFRASTRUCTURE ONLY.  The product path never imports this module.

Primitives: direct 3^3 convolutions with circular padding on NDHWC arrays,
written as a sum over the 27 taps of shifted copies (tap = (dx+1)*9 +
(dy+1)*3 + (dz+1) reads the input at offset (dx, dy, dz)), their gradients,
2^3 average pooling and nearest upsampling with their adjoints, ReLU,
channel concatenation, the 1x1x1 head, the loss (mean squared error in
v = asinh(u / 0.01)) and one Adam step (Kingma & Ba, bias-corrected).

Network (the library's documented learned-start U-Net; not in the paper):
  features x0 = [ln(1 + delta), log10|fR0| + 5, 1, asinh(u_scr / 0.01) / 5,
  0 x 12] with the local screening value u_scr = -(n+1) ln(1 + Om delta /
  Rt) at a = 1 (clamped to [-20, 5]; the arguments of both logarithms
  floored at 1e-3 and 1e-6);
  encoder e_l = relu(conv(relu(conv(p_l)))) with 16/32/64 channels on
  levels 0..2, p_0 = x0, p_{l+1} = avgpool(e_l);
  bottom b = relu(conv(relu(conv(p_3)))) with 128 channels;
  decoder d_l = relu(conv(relu(conv(concat(up(d_{l+1}), e_l))))) (d_3 = b),
  64/32/16 channels on levels 2..0 (up-sampled channels first);
  head v = w . d_0 + c (16 weights, one bias); u = 0.01 sinh(v).
Parameters in one flat FP32 vector: for each of the 14 convolutions in the
order enc0a, enc0b, enc1a, enc1b, enc2a, enc2b, bottom a, bottom b, dec2a,
dec2b, dec1a, dec1b, dec0a, dec0b: W [27][Cin][Cout] then b [Cout]; then
the head's 16 weights and its bias.

With ``bf16=True`` the forward and backward passes round every stored
activation, weight copy and pre-activation gradient to bfloat16 (round to
nearest even) where the library stores them in that format, so that both
sides take those decisions in the same precision; the arithmetic between the
roundings is FP64.  The primitives are pinned in tests/test_nn_oracle.py
(finite differences, explicit loops, closed forms of Adam).
"""
import numpy as np

U_SCALE = 0.01

# (Cin, Cout, level) of the 14 convolutions, in parameter order
CONVS = [(16, 16, 0), (16, 16, 0), (16, 32, 1), (32, 32, 1), (32, 64, 2), (64, 64, 2),
         (64, 128, 3), (128, 128, 3), (192, 64, 2), (64, 64, 2), (96, 32, 1), (32, 32, 1),
         (48, 16, 0), (16, 16, 0)]


def _taps():
    for tap in range(27):
        yield tap, tap // 9 - 1, (tap // 3) % 3 - 1, tap % 3 - 1


def _shift(x, dx, dy, dz):
    """s[b, i, j, k] = x[b, i+dx, j+dy, k+dz] (periodic)."""
    return np.roll(x, shift=(-dx, -dy, -dz), axis=(1, 2, 3))


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), via FP32, returned as FP64."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


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


def avgpool2_bwd(gc):
    """Adjoint of avgpool2: every daughter gets 1/8 of its parent's gradient."""
    return upsample2(gc) / 8.0


def upsample2(x):
    return x.repeat(2, axis=1).repeat(2, axis=2).repeat(2, axis=3)


def upsample2_bwd(gf):
    """Adjoint of upsample2: a parent gets the sum of its 8 daughters' gradients."""
    return 8.0 * avgpool2(gf)


def relu_bwd(g, y):
    """Gradient of the pre-activation from that of y = relu(z): g where y > 0."""
    return np.where(y > 0.0, g, 0.0)


def concat(a, b):
    """Channel concatenation [a, b] (NDHWC)."""
    return np.concatenate([a, b], axis=-1)


def features(delta, fr0_abs, omega_m=0.3, n=1):
    """Network input [D, D, D, 16] for one box at a = 1 (see the module text)."""
    Rt = omega_m + 4.0 * (1.0 - omega_m)
    x = np.zeros(delta.shape + (16,))
    x[..., 0] = np.log(np.maximum(1.0 + delta, 1e-3))
    x[..., 1] = np.log10(fr0_abs) + 5.0
    x[..., 2] = 1.0
    u_scr = np.clip(-(n + 1) * np.log(np.maximum(1.0 + omega_m * delta / Rt, 1e-6)), -20.0, 5.0)
    x[..., 3] = np.arcsinh(u_scr / U_SCALE) / 5.0
    return x


def mse_v(out, u_target):
    """Loss mean((out - asinh(u / U_SCALE))^2) and its gradient w.r.t. out."""
    d = out - np.arcsinh(u_target / U_SCALE)
    return float(np.mean(d * d)), 2.0 * d / d.size


def adam_step(p, g, m1, m2, t, lr, b1=0.9, b2=0.999, eps=1e-8, dtype=np.float64):
    """One Adam step (t = 1, 2, ...): returns (p, m1, m2) after the step."""
    p, g, m1, m2 = (np.asarray(a, dtype=dtype) for a in (p, g, m1, m2))
    one, b1_, b2_ = dtype(1.0), dtype(b1), dtype(b2)
    m1 = b1_ * m1 + (one - b1_) * g
    m2 = b2_ * m2 + (one - b2_) * g * g
    c1 = one - dtype(b1) ** t
    c2 = one - dtype(b2) ** t
    p = p - dtype(lr) * (m1 / c1) / (np.sqrt(m2 / c2) + dtype(eps))
    return p, m1, m2


def param_layout():
    """[(W offset, b offset) per convolution], head offset, total count."""
    offs, off = [], 0
    for ci, co, _ in CONVS:
        offs.append((off, off + 27 * ci * co))
        off += 27 * ci * co + co
    return offs, off, off + 17


def unpack(P):
    offs, hoff, _ = param_layout()
    Ws, bs = [], []
    for (ci, co, _), (wo, bo) in zip(CONVS, offs):
        Ws.append(np.asarray(P[wo:wo + 27 * ci * co], np.float64).reshape(27, ci, co))
        bs.append(np.asarray(P[bo:bo + co], np.float64))
    return Ws, bs, np.asarray(P[hoff:hoff + 16], np.float64), float(P[hoff + 16])


def pack_grads(dWs, dbs, dhw, dhb):
    out = []
    for dW, db in zip(dWs, dbs):
        out += [dW.ravel(), db]
    out += [dhw, np.array([dhb])]
    return np.concatenate(out)


def unet_forward(P, x0, bf16_storage=False):
    """Forward pass; returns (v [B,D,D,D], cache for unet_backward)."""
    r = bf16 if bf16_storage else (lambda a: a)
    Ws, bs, hw, hb = unpack(P)
    Wq = [r(W) for W in Ws]
    acts = {}

    def conv(i, x):
        y = r(conv3d_fwd(x, Wq[i], bs[i], relu=True))
        acts[i] = (x, y)
        return y

    x = r(x0)
    e = []
    p = x
    for lvl in range(3):
        e.append(conv(2 * lvl + 1, conv(2 * lvl, p)))
        p = r(avgpool2(e[-1]))
    d = conv(7, conv(6, p))
    for lvl, i in zip((2, 1, 0), (8, 10, 12)):
        d = conv(i + 1, conv(i, concat(upsample2(d), e[lvl])))
    v = d @ hw + hb
    return v, {"acts": acts, "Wq": Wq, "d0": d, "hw": hw, "e": e}


def unet_backward(cache, gv, bf16_storage=False):
    """Gradient of the flat parameters for the output gradient gv."""
    r = bf16 if bf16_storage else (lambda a: a)
    acts, Wq, hw = cache["acts"], cache["Wq"], cache["hw"]
    dWs, dbs = [None] * 14, [None] * 14
    d0 = cache["d0"]
    dhw = (gv[..., None] * d0).reshape(-1, 16).sum(0)
    dhb = float(gv.sum())
    g = gv[..., None] * hw

    def conv_bwd(i, gy, need_dx=True):
        x, y = acts[i]
        gz = r(relu_bwd(gy, y))
        dWs[i], dbs[i] = conv3d_wgrad(x, gz)
        return conv3d_dgrad(gz, Wq[i]) if need_dx else None

    skip = {}
    for lvl, i, cu in ((0, 12, 32), (1, 10, 64), (2, 8, 128)):
        gcat = conv_bwd(i, conv_bwd(i + 1, g))
        skip[lvl] = gcat[..., cu:]
        g = upsample2_bwd(gcat[..., :cu])
    g = conv_bwd(6, conv_bwd(7, g))  # gradient w.r.t. p_3
    for lvl in (2, 1, 0):
        ge = skip[lvl] + avgpool2_bwd(g)
        g = conv_bwd(2 * lvl, conv_bwd(2 * lvl + 1, ge), need_dx=lvl > 0)
    return pack_grads(dWs, dbs, dhw, dhb)
