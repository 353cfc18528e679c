"""Seeded synthetic inputs for the f(R) solver: lognormal density fields and
Poisson-sampled particles.

This module holds no arithmetic of the method itself; it only draws inputs.
Both the CUDA path (through its callers) and the CPU oracle's tests read the
same arrays from here.  The paper's cosmological snapshots and initial
conditions (Sec. 5) are not available, so these fields stand in for them.

Recipe (all FP64, numpy PCG64):
  g      : unit white noise on N^3, coloured by sqrt(P(k)) with P(k) ~ k^-1.5,
           k = 2 pi |n| / L, the k = 0 mode removed, rescaled to sample std
           sigma_g;
  delta  : exp(g - sigma_g^2 / 2) - 1, then 1 + delta renormalised to mean 1;
  points : per base cell Poisson(nbar (1 + delta)) particles, uniform in the
           cell; order C-order over cells.
Seeds: workload c, realisation r -> 1000 c + r.
"""
from __future__ import annotations

import numpy as np


def gaussian_field(N: int, box: float, sigma_g: float, seed: int, slope: float = -1.5) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    white = rng.standard_normal((N, N, N))
    wk = np.fft.rfftn(white)
    n1 = np.fft.fftfreq(N, d=1.0 / N)
    nz = np.fft.rfftfreq(N, d=1.0 / N)
    kx = n1[:, None, None]
    ky = n1[None, :, None]
    kz = nz[None, None, :]
    kmag = (2.0 * np.pi / box) * np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.zeros_like(kmag)
    nzm = kmag > 0
    amp[nzm] = kmag[nzm] ** (0.5 * slope)
    g = np.fft.irfftn(wk * amp, s=(N, N, N), axes=(0, 1, 2))
    g -= g.mean()
    g *= sigma_g / g.std()
    return g


def lognormal_delta(N: int, box: float, sigma_g: float, seed: int) -> np.ndarray:
    """Lognormal overdensity with mean exactly 0 (float64, shape (N,N,N))."""
    g = gaussian_field(N, box, sigma_g, seed)
    one = np.exp(g - 0.5 * sigma_g * sigma_g)
    one /= one.mean()
    return one - 1.0


def poisson_particles(delta: np.ndarray, box: float, nbar: float, seed: int) -> np.ndarray:
    """Particles Poisson-sampled per cell from nbar (1 + delta), positions
    uniform inside their cell, comoving Mpc/h in [0, box). Shape (Np, 3)."""
    N = delta.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    lam = np.clip(nbar * (1.0 + delta), 0.0, None).ravel()
    counts = rng.poisson(lam)
    cells = np.repeat(np.arange(N * N * N, dtype=np.int64), counts)
    i = cells // (N * N)
    j = (cells // N) % N
    k = cells % N
    off = rng.random((len(cells), 3))
    h = box / N
    pos = np.empty((len(cells), 3))
    pos[:, 0] = (i + off[:, 0]) * h
    pos[:, 1] = (j + off[:, 1]) * h
    pos[:, 2] = (k + off[:, 2]) * h
    np.clip(pos, 0.0, np.nextafter(box, 0.0), out=pos)
    return pos


def workload_seed(workload: int, realisation: int = 0) -> int:
    return 1000 * workload + realisation


# Named workloads (sizes and parameters of the synthetic benchmark cases).
WORKLOADS = {
    "grid32": dict(N=32, box=100.0, a=1.0, fr0=1e-5, sigma_g=1.0, seed=workload_seed(1)),
    "particles256": dict(N=256, box=100.0, a=1.0, fr0=1e-5, sigma_g=1.5, lmax=2, nbar=1.0,
                         seed=workload_seed(2)),
    "particles512": dict(N=512, box=100.0, a=1.0, fr0=1e-6, sigma_g=2.0, lmax=3, nbar=1.0,
                         seed=workload_seed(3)),
}
