"""The power-spectrum analysis of the AMR-vs-fixed-grid comparison (Sec. 5.1),
on the CPU: Parseval's identity over all modes, the white-noise level, and a
single Fourier mode landing in its own |k| bin."""
import numpy as np

from paper_1305_2418_gb300 import enhance


def test_parseval_and_white_noise():
    N, box = 32, 50.0
    rng = np.random.default_rng(0)
    f = rng.standard_normal((N, N, N))
    f -= f.mean()
    k, p, cnt = enhance.power_spectrum(f, box, nbins=10)
    # every mode but k = 0 and the corner modes beyond the Nyquist sphere lands in a
    # bin; with bins up to the Nyquist frequency the sum covers the sphere
    fk = np.fft.fftn(f)
    kk = (2 * np.pi / box) * np.sqrt(sum(np.meshgrid(*[np.fft.fftfreq(N, 1.0 / N) ** 2] * 3,
                                                     indexing="ij")))
    inside = (kk >= 2 * np.pi / box) & (kk <= np.pi * N / box)
    want = (np.abs(fk[inside]) ** 2).sum() * box ** 3 / N ** 6
    assert abs((p * cnt).sum() / want - 1.0) < 1e-12
    # white noise: P = variance x cell volume on average
    h3 = (box / N) ** 3
    assert abs(np.average(p, weights=cnt) / (f.var() * h3) - 1.0) < 0.05


def test_single_mode():
    N, box = 32, 40.0
    x = np.arange(N) * box / N
    m = 5
    f = np.broadcast_to(np.cos(2 * np.pi * m * x / box)[:, None, None], (N, N, N)).copy()
    k, p, cnt = enhance.power_spectrum(f, box, nbins=12)
    kmode = 2 * np.pi * m / box
    top = np.argmax(p)
    assert 0 < top < len(k) - 1 and k[top - 1] < kmode < k[top + 1]
    assert p[top] > 1e10 * np.delete(p, top).max()
