"""The seeded synthetic inputs follow their stated recipe: a Gaussian field
with the requested sample std and a k^-1.5 spectrum, a lognormal delta with
mean exactly 0, and Poisson particles inside their cells with the expected
counts; equal seeds give equal arrays.  CPU only."""
import numpy as np

from paper_1305_2418_gb300 import synth


def test_gaussian_field_std_mean_and_spectral_slope():
    N, box = 64, 100.0
    g = synth.gaussian_field(N, box, 1.3, 11)
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 1.3) < 1e-12
    # spectral slope: shell-averaged |g_k|^2 against |k| over the resolved band
    p = np.abs(np.fft.rfftn(g)) ** 2
    n1 = np.fft.fftfreq(N, d=1.0 / N)
    nz = np.fft.rfftfreq(N, d=1.0 / N)
    kk = np.sqrt(n1[:, None, None] ** 2 + n1[None, :, None] ** 2 + nz[None, None, :] ** 2)
    shells = np.arange(2, N // 2)
    pk = np.array([p[(kk >= s - 0.5) & (kk < s + 0.5)].mean() for s in shells])
    slope = np.polyfit(np.log(shells), np.log(pk), 1)[0]
    assert abs(slope + 1.5) < 0.1, slope
    assert p[0, 0, 0] < 1e-18 * p.sum()  # the k = 0 mode is removed


def test_lognormal_delta_mean_zero_and_positive_density():
    d = synth.lognormal_delta(32, 100.0, 1.5, 12)
    assert d.shape == (32, 32, 32)
    assert abs(d.mean()) < 1e-14
    assert (1.0 + d).min() > 0.0
    np.testing.assert_array_equal(d, synth.lognormal_delta(32, 100.0, 1.5, 12))
    assert not np.array_equal(d, synth.lognormal_delta(32, 100.0, 1.5, 13))


def test_poisson_particles_in_their_cells_with_expected_counts():
    N, box, nbar = 16, 50.0, 3.0
    d = synth.lognormal_delta(N, box, 1.0, 14)
    pos = synth.poisson_particles(d, box, nbar, 14)
    assert pos.shape[1] == 3 and pos.min() >= 0.0 and pos.max() < box
    # total count within a few Poisson standard deviations of nbar N^3
    expect = nbar * N ** 3
    assert abs(len(pos) - expect) < 5.0 * np.sqrt(expect)
    # particles come cell by cell in C order, each inside its cell
    h = box / N
    idx = np.floor(pos / h).astype(np.int64)
    lin = (idx[:, 0] * N + idx[:, 1]) * N + idx[:, 2]
    assert np.all(np.diff(lin) >= 0)
    counts = np.bincount(lin, minlength=N ** 3)
    lam = nbar * (1.0 + d.ravel())
    # the per-cell counts follow Poisson(lam): mean and variance of (n - lam)
    r = counts - lam
    assert abs(r.mean()) < 5.0 * np.sqrt(lam.mean() / N ** 3)
    assert abs(r.var() / lam.mean() - 1.0) < 0.1
    np.testing.assert_array_equal(pos, synth.poisson_particles(d, box, nbar, 14))


def test_named_workloads_and_seeds():
    w = synth.WORKLOADS["particles256"]
    assert (w["N"], w["lmax"], w["nbar"], w["sigma_g"], w["fr0"]) == (256, 2, 1.0, 1.5, 1e-5)
    assert synth.workload_seed(2, 3) == 2003
