"""Enhancement of gravity as a function of scale, from fixed grids and from
the refined hierarchy (the test of Sec. 5.1): the ratio of the power spectrum
of delta + delta_eff to that of delta (Eqs. (30)-(31)).

The field solves, the effective density and its assignment to the PM grid run
in the library (mgfr_solve_particles, mgfr_pm_potential with the matter
density returned, mgfr_effective_mass_pm).  The power spectra are analysis of
the library's outputs, done here with numpy FFTs on the host: shell averages
of |FFT|^2 in bins of |k|.
"""
from __future__ import annotations

import numpy as np

from . import mgfr


def power_spectrum(field: np.ndarray, box: float, nbins: int = 24):
    """(k centres [h/Mpc], P(k), modes per bin) of a periodic N^3 field in
    logarithmic |k| bins from the fundamental to the Nyquist frequency."""
    N = field.shape[0]
    fk = np.fft.rfftn(field)
    p = (fk.real ** 2 + fk.imag ** 2) * (box ** 3 / float(N) ** 6)
    n1 = np.fft.fftfreq(N, d=1.0 / N)
    nz = np.fft.rfftfreq(N, d=1.0 / N)
    kmag = (2.0 * np.pi / box) * np.sqrt(n1[:, None, None] ** 2 + n1[None, :, None] ** 2 +
                                         nz[None, None, :] ** 2)
    # rfft halves the z axis: modes with 0 < kz < N/2 stand for two
    w = np.full(nz.shape, 2.0)
    w[0] = 1.0
    if N % 2 == 0:
        w[-1] = 1.0
    w = np.broadcast_to(w[None, None, :], kmag.shape)
    kf, kn = 2.0 * np.pi / box, np.pi * N / box
    edges = np.logspace(np.log10(kf), np.log10(kn), nbins + 1)
    kr = kmag.ravel()
    idx = np.searchsorted(edges, kr, side="right") - 1
    idx[np.abs(kr - kn) <= 1e-12 * kn] = nbins - 1  # Nyquist modes close the last bin
    idx[np.abs(kr - kf) <= 1e-12 * kf] = 0
    ok = (idx >= 0) & (idx < nbins)
    cnt = np.bincount(idx[ok], weights=w.ravel()[ok], minlength=nbins)
    ps = np.bincount(idx[ok], weights=(w * p).ravel()[ok], minlength=nbins)
    ks = np.bincount(idx[ok], weights=(w * kmag).ravel()[ok], minlength=nbins)
    good = cnt > 0
    return ks[good] / cnt[good], ps[good] / cnt[good], cnt[good]


def run(pos, box: float, fr0: float, N_base: int, max_level: int, N_pm: int,
        precision: int = mgfr.PREC_MIXED, a: float = 1.0, device: int = 0, nbins: int = 24):
    """One solve of the particles `pos` ([Np, 3] CUDA FP64) on an N_base grid
    with max_level refinement levels, then delta and delta_eff on the periodic
    PM grid of N_pm cells per axis.  Returns (k, P(delta + delta_eff) /
    P(delta), P(delta), solve stats)."""
    lpm = int(round(np.log2(N_pm // N_base)))
    assert N_base << lpm == N_pm
    s = mgfr.Solver(device, fr0_abs=fr0, precision=precision, max_level=max_level)
    out = s.solve_particles(pos, N_base, box, a, want_fr=False, want_acc=False)
    _, dens, _ = s.pm_potential(N_base, lpm, mgfr.PM_MATTER, want_density=True)
    eff = s.effective_mass_pm(N_base, lpm)
    d = dens.cpu().numpy()
    e = eff.cpu().numpy()
    s.close()
    k, p_m, _ = power_spectrum(d, box, nbins)
    _, p_t, _ = power_spectrum(d + e, box, nbins)
    return k, p_t / p_m, p_m, out["stats"]
