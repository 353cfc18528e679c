"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, an exact solution of the linearised discrete problem by FFT, a dense
Newton solve with a numerically differentiated Jacobian, a number the paper
prints, brute force on tiny inputs, or an invariant.  CPU only.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1305_2418_gb300 import synth

C_OVER_H0 = 2997.92458  # c / H0 in Mpc/h
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def paper_background(fr0_abs, a, omega_m=0.3, n=1):
    """R_bar(a) in units of H0^2 and fR_bar(a) (Sec. 2, Eq. (10)), flat LCDM."""
    ol = 1.0 - omega_m
    R = 3.0 * omega_m * (a ** -3 + 4.0 * ol / omega_m)
    R0 = 3.0 * omega_m * (1.0 + 4.0 * ol / omega_m)
    return R, -fr0_abs * (R0 / R) ** (n + 1)


def discrete_k2(N, box):
    """Eigenvalues of the 7-point periodic Laplacian (and sin(k h)/h per axis)."""
    h = box / N
    k1 = 2.0 * np.pi * np.fft.fftfreq(N, d=h)
    lam = (2.0 - 2.0 * np.cos(k1 * h)) / h ** 2
    k2 = lam[:, None, None] + lam[None, :, None] + lam[None, None, :]
    return k2, np.sin(k1 * h) / h


# --------------------------------------------------------------------------
# P1: no perturbation -> background solution u = 0 (Sec. 3.2: L(0) = 0).
# --------------------------------------------------------------------------
def test_background_solution_from_nonzero_start():
    N = 16
    rng = np.random.default_rng(5)
    u0 = 0.1 * rng.standard_normal((N, N, N))
    u, st = oracle.solve_dense(np.zeros((N, N, N)), 100.0, 1e-5, u0=u0, tol=1e-13)
    assert st["converged"] == 1.0
    assert np.abs(u).max() < 1e-12


# --------------------------------------------------------------------------
# P2: small perturbations -> exact FFT solution of the linearised discrete
# equation.  The linear coefficients come from the paper's own formulas:
# Yukawa mass lambda^2 = (1/3c^2) dR/dfR at fR_bar (Sec. 4.1) and the source
# 8 pi G rho_bar = 3 H0^2 Om a^-3; comoving lengths multiply by a.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("fr0,a", [(1e-5, 1.0), (1e-4, 1.0), (1e-5, 0.5)])
def test_linear_limit_matches_fft_helmholtz(fr0, a):
    N, box, om = 32, 100.0, 0.3
    delta = 1e-6 * synth.lognormal_delta(N, box, 1.0, 4242)
    Rbar, fbar = paper_background(fr0, a, om)
    kappa = 1.0 / C_OVER_H0 ** 2
    # dR/dfR from delta R = R_bar (sqrt(fR_bar / fR) - 1)  (Eq. (11))
    dRdf = Rbar / (2.0 * abs(fbar))
    mu2 = a * a * kappa * dRdf / 3.0
    S = a * a * kappa * om * a ** -3 / abs(fbar)
    k2, sk = discrete_k2(N, box)
    uh = -S * np.fft.fftn(delta) / (k2 + mu2)
    u_fft = np.real(np.fft.ifftn(uh))
    # rounding of 1 - exp(-u/2) at |u| ~ 1e-7 floors the relative residual near 1e-10
    u, st = oracle.solve_dense(delta, box, fr0, a=a, tol=1e-9, omega_m=om)
    assert st["converged"] == 1.0
    err = np.abs(u - u_fft).max() / np.abs(u_fft).max()
    assert err < 1e-5, err
    # Force: a_MG / c^2 = grad fR / (2a), central difference = i sin(kh)/h.
    fr_fft = fbar * np.exp(u_fft)
    Fk = np.fft.fftn(fr_fft)
    g = [np.real(np.fft.ifftn(1j * sk[:, None, None] * Fk)),
         np.real(np.fft.ifftn(1j * sk[None, :, None] * Fk)),
         np.real(np.fft.ifftn(1j * sk[None, None, :] * Fk))]
    acc_fft = np.stack(g) / (2.0 * a)
    fr, acc = oracle.force_dense(u, box, fr0, a=a, omega_m=om)
    assert np.abs(fr / fr_fft - 1.0).max() < 1e-10
    aerr = np.abs(acc - acc_fft).max() / np.abs(acc_fft).max()
    assert aerr < 1e-5, aerr


# --------------------------------------------------------------------------
# P3: brute-force dense Newton on 8^3.  F(u) = L(u) - f is written here with
# array shifts, its Jacobian taken by complex-step differentiation (exact to
# rounding, independent of any hand-written derivative) and the Newton steps
# solved by LAPACK.
# --------------------------------------------------------------------------
def _F(u, f, h, alpha, Rt, n):
    E = np.exp(u)
    lap = 0.0
    for ax in range(3):
        for s in (1, -1):
            un = np.roll(u, s, axis=ax)
            lap = lap + 0.5 * (np.exp(un) + E) * (un - u)
    return lap / h ** 2 + alpha * Rt * (1.0 - np.exp(-u / (n + 1))) - f


@pytest.mark.parametrize("fr0", [1e-5, 1e-6])
def test_dense_newton_8cubed(fr0):
    N, box, om, a, n = 8, 25.0, 0.3, 1.0, 1
    delta = synth.lognormal_delta(N, box, 1.0, 77)
    Rbar, fbar = paper_background(fr0, a, om)
    Rt = Rbar / 3.0
    alpha = a * a / C_OVER_H0 ** 2 / fbar
    f = -alpha * om * delta
    h = box / N
    u = -2.0 * np.log1p(om * delta / Rt)  # local-screening start
    for _ in range(60):
        Fu = _F(u, f, h, alpha, Rt, n)
        if np.abs(Fu).max() < 1e-13 * np.abs(f).max():
            break
        J = np.empty((N ** 3, N ** 3))
        hs = 1e-30
        for j in range(N ** 3):
            du = np.zeros(N ** 3, dtype=complex)
            du[j] = 1j * hs
            J[:, j] = np.imag(_F(u + du.reshape(u.shape), f, h, alpha, Rt, n)).ravel() / hs
        step = np.linalg.solve(J, -Fu.ravel()).reshape(u.shape)
        t = 1.0
        while np.abs(_F(u + t * step, f, h, alpha, Rt, n)).max() > np.abs(Fu).max() and t > 1e-4:
            t *= 0.5
        u = u + t * step
    assert np.abs(_F(u, f, h, alpha, Rt, n)).max() < 1e-13 * np.abs(f).max()
    uo, st = oracle.solve_dense(delta, box, fr0, tol=1e-13, max_vcycles=200)
    assert st["converged"] == 1.0
    assert np.abs(uo - u).max() < 1e-9


# --------------------------------------------------------------------------
# P4: manufactured solutions.  f := L(u*) for a chosen u*; the discrete
# solution is u* itself (unique: -L is monotone in u), so the solver must
# return it, also in the stiff regime (u* down to -8).
# --------------------------------------------------------------------------
@pytest.mark.parametrize("offset,amp,fr0", [(0.0, 0.5, 1e-5), (-4.0, 4.0, 1e-6)])
def test_manufactured_solution(offset, amp, fr0):
    N, box = 32, 100.0
    x = (np.arange(N) + 0.5) * box / N
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    g = synth.gaussian_field(N, box, 1.0, 9)
    ustar = offset + amp * np.sin(2 * np.pi * X / box) * np.cos(4 * np.pi * Y / box) + 0.2 * g
    f = oracle.apply_L_dense(ustar, box, fr0)
    u, st = oracle.solve_dense(None if False else np.zeros_like(ustar), box, fr0, f=f, tol=1e-12,
                               max_vcycles=200)
    assert st["converged"] == 1.0
    assert np.abs(u - ustar).max() < 1e-8


# --------------------------------------------------------------------------
# P5: the paper's 1D density peak (Sec. 4.2, Eq. (36)).
# (a) The printed amplitude A ~ 2.7e-5 follows from mean(delta rho) = 0 and
#     delta R(fR) of Eq. (11): A = |fR_bar| mean((1 - alpha e^{-x^2/w^2})^{-1/2})^2.
# (b) With a resolved peak the discrete solution converges to the analytic
#     fR at second order in the cell size.
# --------------------------------------------------------------------------
def test_peak_amplitude_matches_paper():
    """The oracle's discrete operator reproduces the printed amplitude.

    Summed over a periodic grid, the flux terms of L cancel pairwise, so
    sum_i L_i(u) = alpha Rt sum_i (1 - e^{-u_i/(n+1)}) for any field, and
    mean(delta rho) = 0 (mean f = 0) is sum_i L_i(u) = 0.  The field u of
    Eq. (36) is sampled at 64^3 points spaced 0.001 Mpc/h along x (the core of
    width w sqrt(1 - alpha) ~ 0.05 Mpc/h is resolved) and laid out on a 64^3
    grid; the A for which the oracle's sum of L vanishes must be the paper's
    A ~ 2.7e-5.  The same root with the exponent of n = 2 lands far away, so
    the pin sees the 1/(n+1) of the nonlinear term."""
    from scipy.optimize import brentq
    with open(os.path.join(GOLDEN, "peak1d_amplitude.json")) as fh:
        gold = json.load(fh)
    L, w, al, fb = gold["box"], gold["w"], gold["alpha"], gold["fr_bar_abs"]
    N = 64
    M = N ** 3
    x = (np.arange(M) + 0.5) * (L / M) - L / 2
    e = np.exp(-x * x / w ** 2)

    def total_L(A, n=1):
        u = np.log((A / fb) * (1.0 - al * e)).reshape(N, N, N)
        return float(oracle.apply_L_dense(u, L, fb, n=n).sum())

    A = brentq(total_L, 1e-6, 1e-3, xtol=1e-12)
    assert abs(A - gold["A"]) <= gold["tol"], A
    # the oracle's mean source is zero there: mean delta rho = 0
    u = np.log((A / fb) * (1.0 - al * e)).reshape(N, N, N)
    mc = oracle.model_constants(fb)
    f = oracle.apply_L_dense(u, L, fb)
    assert abs(f.mean() / (mc["alpha"] * 0.3)) < 1e-9
    A2 = brentq(lambda a_: total_L(a_, n=2), 1e-7, 1e-3, xtol=1e-12)
    assert abs(A2 - gold["A"]) > 5 * gold["tol"], A2


def _peak_delta(N, box, w, al, fb, om):
    x = (np.arange(N) + 0.5) * box / N - box / 2
    from scipy.integrate import quad
    M, _ = quad(lambda s: (1.0 - al * np.exp(-s * s / w ** 2)) ** -0.5, -box / 2, box / 2,
                points=[0.0], limit=500)
    A = fb * (M / box) ** 2
    e = np.exp(-x * x / w ** 2)
    fr = -A * (1.0 - al * e)
    frpp = -(2.0 * A * al / w ** 2) * (1.0 - 2.0 * x * x / w ** 2) * e
    Rt = (3.0 * om * (1 + 4 * (1 - om) / om)) / 3.0  # R_bar / (3 H0^2) at a = 1
    # 8 pi G delta rho = delta R - 3 c^2 fR''; in H0 = 1 units, a = 1.
    d1 = (3.0 * Rt * (np.sqrt(-fb / fr) - 1.0) - 3.0 * C_OVER_H0 ** 2 * frpp) / (3.0 * om)
    u1 = np.log(fr / -fb)
    delta = np.broadcast_to(d1[:, None, None], (N, N, N)).copy()
    return delta, u1


def test_peak_converges_second_order():
    box, w, al, fb, om = 128.0, 15.0, 0.9, 1e-5, 0.3
    errs = []
    for N in (32, 64):
        delta, u1 = _peak_delta(N, box, w, al, fb, om)
        u, st = oracle.solve_dense(delta, box, fb, tol=1e-11)
        assert st["converged"] == 1.0
        assert np.abs(u - u[:, :1, :1]).max() < 1e-10  # stays one-dimensional
        errs.append(np.abs(u[:, 0, 0] - u1).max())
    assert errs[1] < 0.35 * errs[0], errs
    assert errs[1] < 0.05, errs


# --------------------------------------------------------------------------
# P6: screened interior.  Where delta is uniform over a region much wider than
# the Compton length, lap e^u -> 0 and u = -(n+1) ln(1 + Om a^-3 delta / Rt).
# --------------------------------------------------------------------------
def test_screened_tophat_interior():
    N, box, R, din, fr0, om = 32, 100.0, 20.0, 10.0, 1e-6, 0.3
    x = (np.arange(N) + 0.5) * box / N - box / 2
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    inside = X ** 2 + Y ** 2 + Z ** 2 < R * R
    dbg = -din * inside.sum() / (~inside).sum()
    delta = np.where(inside, din, dbg)
    u, st = oracle.solve_dense(delta, box, fr0, tol=1e-12)
    assert st["converged"] == 1.0
    Rt = om + 4 * (1 - om)
    uc_exact = -2.0 * np.log1p(om * din / Rt)
    ub_exact = -2.0 * np.log1p(om * dbg / Rt)
    c = N // 2
    assert abs(u[c, c, c] / uc_exact - 1.0) < 1e-6
    assert abs(u[0, 0, 0] / ub_exact - 1.0) < 1e-4
    # unscreened (|fR0| = 1e-4, small delta) is covered by the FFT pin above.


# --------------------------------------------------------------------------
# Effective mass density (Sec. 2.4): delta_eff = delta/3 - delta R/(24 pi G rho)
# with delta R from Eq. (11).  Unscreened limits give the 1/3 enhancement,
# full screening gives 0 (GR), and on a converged periodic solve the box sum
# is fixed by the discrete equation itself.
# --------------------------------------------------------------------------
def test_effective_density_limits_and_box_sum():
    rng = np.random.default_rng(9)
    d = rng.standard_normal((8, 8, 8))
    # u = 0 (f_R at its background value): delta R = 0, delta_eff = delta / 3
    np.testing.assert_allclose(oracle.effective_density(np.zeros_like(d), d, 1e-5), d / 3.0,
                               rtol=0, atol=1e-15)
    # local screening, u = -(n+1) ln(1 + Om a^-3 delta / Rt): delta_eff = 0, any a and n
    for a, n in ((1.0, 1), (0.5, 1), (1.0, 2)):
        mc = oracle.model_constants(1e-5, a=a, n=n)
        dd = np.abs(d) * 5.0
        u = -(n + 1) * np.log1p(0.3 / a ** 3 * dd / mc["Rt"])
        eff = oracle.effective_density(u, dd, 1e-5, a=a, n=n)
        assert np.abs(eff).max() < 1e-13 * np.abs(dd).max()
    # converged periodic solve: the divergence term sums to zero, so
    # sum(L) = alpha Rt sum(1 - e^{-u/2}) = sum(f) - sum(r), i.e.
    # sum(delta_eff) = -sum(r) / (3 alpha Om a^-3) whatever sum(delta) is (a
    # mean of 0.2 here, so that a wrong coefficient would show)
    N, box, fr0 = 16, 50.0, 1e-5
    delta = synth.lognormal_delta(N, box, 1.5, 90) + 0.2
    u, st = oracle.solve_dense(delta, box, fr0, tol=1e-12)
    assert st["converged"] == 1.0
    r = oracle.residual_dense(u, delta, box, fr0)
    mc = oracle.model_constants(fr0)
    eff = oracle.effective_density(u, delta, fr0)
    want = -r.sum() / (3.0 * mc["alpha"] * 0.3)
    assert abs(eff.sum() - want) < 1e-9 * np.abs(eff).sum()
    assert abs(delta.sum() / 3.0) > 1e3 * abs(eff.sum())
    # (delta R is not negligible here: the case is not the u = 0 limit)
    assert np.abs(eff - delta / 3.0).max() > 1e-2 * np.abs(delta / 3.0).max()


def _leaf_effective_by_brute_force(A, L, a=1.0, n=1, fr0=1e-5, matter=False):
    """delta_eff (or, with matter=True, delta) sampled at every cell of the
    uniform level-L grid, from the leaf that contains it (found by descending
    the hierarchy cell by cell)."""
    N0 = A.N0
    NL = N0 << L
    if matter:
        eff = [A.delta(l) for l in range(A.nlev)]
    else:
        eff = [oracle.effective_density(A.u(l), A.delta(l), fr0, a=a, n=n)
               for l in range(A.nlev)]
    keys = [None] + [A.keys(l) for l in range(1, A.nlev)]
    out = np.empty((NL, NL, NL))
    for i in range(NL):
        for j in range(NL):
            for k in range(NL):
                for l in range(A.nlev):
                    sh = L - l
                    I, J, K = i >> sh, j >> sh, k >> sh
                    Nl = N0 << l
                    if l == 0:
                        c = (I * Nl + J) * Nl + K
                    else:
                        Np = Nl // 2
                        key = ((I >> 1) * Np + (J >> 1)) * Np + (K >> 1)
                        o = np.searchsorted(keys[l], key)
                        c = 8 * o + ((I & 1) << 2) + ((J & 1) << 1) + (K & 1)
                    if l == A.nlev - 1 or not A.refined(l)[c]:
                        out[i, j, k] = eff[l][c]
                        break
    return out


def test_effective_mass_on_pm_grid_matches_brute_force():
    """Sec. 2.4 long-range part: each leaf's effective mass shared among the
    PM cells it overlaps by volume.  Against sampling the leaf field on the
    finest grid and averaging it over each PM cell, for PM grids coarser
    than, equal to and finer than the leaves; the total is conserved."""
    N0, box, fr0 = 8, 20.0, 1e-5
    rng = np.random.default_rng(21)
    pos = np.concatenate([4.0 + 3.0 * rng.random((600, 3)), box * rng.random((200, 3))])
    A = oracle.AMR(pos, N0, box, 2, 8)
    assert A.nlev == 3
    A.deposit()
    A.set_model(fr0)
    for l in range(A.nlev):
        A.set_u(l, 0.5 * rng.standard_normal(A.ncell(l)))
    fine = _leaf_effective_by_brute_force(A, 2, fr0=fr0)
    for lpm in (0, 1, 2, 3):
        pm = A.effective_pm(lpm)
        Npm = N0 << lpm
        if lpm <= 2:
            s = 1 << (2 - lpm)
            want = fine.reshape(Npm, s, Npm, s, Npm, s).mean(axis=(1, 3, 5))
        else:
            want = np.repeat(np.repeat(np.repeat(fine, 2, 0), 2, 1), 2, 2)
        np.testing.assert_allclose(pm, want, rtol=1e-12, atol=1e-12)
        assert abs(pm.mean() - fine.mean()) < 1e-12
    # no refinement: the PM field is the base level's delta_eff itself
    B = oracle.AMR(pos, N0, box, 0, 8)
    B.deposit()
    B.set_model(fr0)
    u0 = 0.3 * rng.standard_normal(B.ncell(0))
    B.set_u(0, u0)
    np.testing.assert_array_equal(B.effective_pm(0).ravel(),
                                  oracle.effective_density(u0, B.delta(0), fr0))


def test_matter_and_total_on_pm_grid():
    """The matter contrast goes to the PM grid by the same volume shares as
    the effective mass (against brute-force sampling of the leaf field); on
    the base grid it is the base level's delta (ancestors hold the sums of
    their leaves); the total is the sum of the two (Eq. (30))."""
    N0, box, fr0 = 8, 20.0, 1e-5
    rng = np.random.default_rng(22)
    pos = np.concatenate([4.0 + 3.0 * rng.random((600, 3)), box * rng.random((200, 3))])
    A = oracle.AMR(pos, N0, box, 2, 8)
    A.deposit()
    A.set_model(fr0)
    for l in range(A.nlev):
        A.set_u(l, 0.5 * rng.standard_normal(A.ncell(l)))
    fine = _leaf_effective_by_brute_force(A, 2, fr0=fr0, matter=True)
    for lpm in (0, 1, 2, 3):
        pm = A.density_pm(lpm, 1)
        Npm = N0 << lpm
        if lpm <= 2:
            s = 1 << (2 - lpm)
            want = fine.reshape(Npm, s, Npm, s, Npm, s).mean(axis=(1, 3, 5))
        else:
            want = np.repeat(np.repeat(np.repeat(fine, 2, 0), 2, 1), 2, 2)
        np.testing.assert_allclose(pm, want, rtol=1e-12, atol=1e-12)
        assert abs(pm.mean()) < 1e-12  # the particle mass is conserved
        np.testing.assert_allclose(A.density_pm(lpm, 2), pm + A.effective_pm(lpm), rtol=0,
                                   atol=1e-12)
    np.testing.assert_allclose(A.density_pm(0, 1).ravel(), A.delta(0), rtol=0, atol=1e-12)


def test_pm_potential_scale_from_the_field_identity():
    """The potential of the effective mass is -(c^2/2) f_R up to a constant
    (Sec. 2.4: Eqs. (13) and (30) give the same force): with the Poisson
    scale (3/2) Om H0^2 / a of the PM potential the oracle's phi of
    delta_eff matches -(c^2/2)(f_R - mean f_R) to the square of the link
    differences, at a = 1 and a = 0.5."""
    c = 299792.458
    N0, box, fr0 = 16, 100.0, 1e-4
    d = synth.lognormal_delta(N0, box, 0.3, 96)
    pos = synth.poisson_particles(d, box, 64.0, 97)
    for a in (1.0, 0.5):
        A = oracle.AMR(pos, N0, box, 0, 8)
        A.deposit()
        A.set_model(fr0, a=a)
        rc, _ = A.solve(tol=1e-13)
        assert rc == 0
        u = A.u(0)
        fr = oracle.model_constants(fr0, a=a)["fbar"] * np.exp(u)
        want = -0.5 * c * c * (fr - fr.mean())
        got = A.pm_potential(0, what=0).ravel()
        uu = u.reshape((N0,) * 3)
        links = max(np.abs(np.diff(uu, axis=ax)).max() for ax in range(3))
        assert links > 1e-3
        err = np.abs(got - want).max() / np.abs(want).max()
        assert err < 0.5 * links * links, (a, err, links)
        A.close()


def test_pm_accel_central_difference_and_cic():
    """The PM force: the central difference of a sine is its exact discrete
    derivative, and the cloud-in-cell interpolation equals scipy's periodic
    trilinear interpolation (map_coordinates, order 1, grid-wrap) of the same
    cell-centred field."""
    from scipy.ndimage import map_coordinates
    N, box = 16, 40.0
    h = box / N
    x = (np.arange(N) + 0.5) * h
    k = 2.0 * np.pi * 3 / box
    phi = np.broadcast_to(np.sin(k * x)[:, None, None], (N, N, N)).copy()
    rng = np.random.default_rng(41)
    pos = box * rng.random((300, 3))
    acc = oracle.pm_accel(phi, box, pos)
    # g_x at cell centres is -cos(k x) sin(k h) / h exactly; at particles the
    # interpolation of it
    gx = -np.cos(k * x) * np.sin(k * h) / h
    gfield = np.broadcast_to(gx[:, None, None], (N, N, N))
    coords = (pos / h - 0.5).T
    want = map_coordinates(gfield, coords, order=1, mode="grid-wrap")
    np.testing.assert_allclose(acc[:, 0], want, rtol=0, atol=1e-13 * np.abs(gx).max())
    assert np.abs(acc[:, 1:]).max() < 1e-13 * np.abs(gx).max()
    # a general field, every component
    phi = rng.standard_normal((N, N, N))
    acc = oracle.pm_accel(phi, box, pos)
    for d in range(3):
        g = -(np.roll(phi, -1, d) - np.roll(phi, 1, d)) / (2 * h)
        want = map_coordinates(g, coords, order=1, mode="grid-wrap")
        np.testing.assert_allclose(acc[:, d], want, rtol=1e-12, atol=1e-12)


def _lap7(phi, box):
    h = box / phi.shape[0]
    out = -6.0 * phi
    for ax in range(3):
        out += np.roll(phi, 1, ax) + np.roll(phi, -1, ax)
    return out / (h * h)


def test_periodic_poisson_inverts_the_seven_point_laplacian():
    rng = np.random.default_rng(31)
    phi = rng.standard_normal((16, 16, 16))
    phi -= phi.mean()
    got = oracle.poisson_periodic(_lap7(phi, 40.0), 40.0)
    assert np.abs(got - phi).max() < 1e-11 * np.abs(phi).max()
    # a constant right-hand side has no periodic solution: its mean is dropped
    got = oracle.poisson_periodic(_lap7(phi, 40.0) + 3.0, 40.0)
    assert np.abs(got - phi).max() < 1e-11 * np.abs(phi).max()


def test_effective_mass_potential_reproduces_the_field():
    """With delta R from Eq. (11) the field equation reads lap f_R =
    -3 a^2 (H0/c)^2 Om a^-3 delta_eff (Sec. 2.4), so the potential of the
    effective mass is -(c^2/2) f_R: the Poisson solve of delta_eff gives back
    E = e^u up to its mean.  The discrete operator's flux 1/2 (E_j + E_i)
    (u_j - u_i) differs from E_j - E_i by -E_i (u_j - u_i)^3 / 12 + ..., so on
    a mildly nonlinear field the two agree to the square of the link
    differences."""
    N, box, fr0 = 16, 100.0, 1e-4
    delta = synth.lognormal_delta(N, box, 0.3, 95)
    u, st = oracle.solve_dense(delta, box, fr0, tol=1e-13)
    assert st["converged"] == 1.0
    mc = oracle.model_constants(fr0)
    eff = oracle.effective_density(u, delta, fr0)
    E = np.exp(u)
    got = oracle.poisson_periodic(-3.0 * mc["alpha"] * 0.3 * eff, box)
    var = E - E.mean()
    links = max(np.abs(np.diff(u, axis=ax)).max() for ax in range(3))
    assert links > 1e-3  # not the linear limit
    err = np.abs(got - var).max() / np.abs(var).max()
    assert err < 0.5 * links * links, (err, links)


# --------------------------------------------------------------------------
# P7: invariants of the discrete problem and independence of accelerators.
# --------------------------------------------------------------------------
def test_shift_and_permutation_invariance():
    N, box = 16, 50.0
    d = synth.lognormal_delta(N, box, 1.2, 31)
    u, _ = oracle.solve_dense(d, box, 1e-5, tol=1e-12)
    us, _ = oracle.solve_dense(np.roll(d, (2, 4, 6), axis=(0, 1, 2)), box, 1e-5, tol=1e-12)
    assert np.abs(np.roll(us, (-2, -4, -6), axis=(0, 1, 2)) - u).max() < 1e-10
    up, _ = oracle.solve_dense(d.transpose(2, 0, 1).copy(), box, 1e-5, tol=1e-12)
    assert np.abs(up.transpose(1, 2, 0) - u).max() < 1e-10


def test_accelerator_independence():
    N, box = 32, 100.0
    d = synth.lognormal_delta(N, box, 1.5, 32)
    ref, _ = oracle.solve_dense(d, box, 1e-5, tol=1e-12)
    for kw in (dict(prolong_linear=False), dict(n_pre=1, n_post=1), dict(n_pre=3, n_post=2),
               dict(step_cap=0.5)):
        u, st = oracle.solve_dense(d, box, 1e-5, tol=1e-12, max_vcycles=300, **kw)
        assert st["converged"] == 1.0, kw
        assert np.abs(u - ref).max() < 1e-9, kw


def test_gradient_sums_to_zero_on_periodic_level():
    N, box = 16, 50.0
    d = synth.lognormal_delta(N, box, 1.0, 33)
    u, _ = oracle.solve_dense(d, box, 1e-5, tol=1e-10)
    fr, acc = oracle.force_dense(u, box, 1e-5)
    assert np.abs(acc.reshape(3, -1).sum(1)).max() < 1e-12 * np.abs(acc).max() * N ** 3


# --------------------------------------------------------------------------
# Refinement structure (Sec. 3.1): brute force with dense masks per level.
# --------------------------------------------------------------------------
def _brute_structure(pos, N0, box, lmax, thr, want_exists=False):
    t = pos * (N0 / box)
    exists = [np.ones((N0,) * 3, bool)]
    keys = [None]
    for l in range(lmax):
        Nl = N0 << l
        idx = np.floor(t * 2 ** l).astype(np.int64)
        cnt = np.zeros((Nl,) * 3, np.int64)
        np.add.at(cnt, (idx[:, 0], idx[:, 1], idx[:, 2]), 1)
        cnt *= exists[l]
        flag = (cnt > thr) & exists[l]
        dil = np.zeros_like(flag)
        for a in (-1, 0, 1):
            for b in (-1, 0, 1):
                for c in (-1, 0, 1):
                    dil |= np.roll(flag, (a, b, c), axis=(0, 1, 2))
        ref = dil & exists[l]
        if not ref.any():
            break
        keys.append(np.flatnonzero(ref.ravel()))
        ex = np.repeat(np.repeat(np.repeat(ref, 2, 0), 2, 1), 2, 2)
        exists.append(ex)
    return (keys, exists) if want_exists else keys


def _brute_leaf_levels(pos, N0, box, exists):
    """Level of the deepest existing cell holding each particle (Sec. 3.1:
    the AMR cell a particle resides in), from the dense existence masks."""
    t = pos * (N0 / box)
    lev = np.zeros(len(pos), np.int64)
    for l in range(1, len(exists)):
        idx = np.floor(t * 2 ** l).astype(np.int64)
        inside = exists[l][idx[:, 0], idx[:, 1], idx[:, 2]]
        lev[inside] = l
    return lev


@pytest.mark.parametrize("N0,lmax,sig,thr", [(16, 2, 1.5, 8), (16, 3, 2.0, 2), (8, 2, 1.0, 0)])
def test_structure_matches_brute_force(N0, lmax, sig, thr):
    box = 100.0
    d = synth.lognormal_delta(N0, box, sig, 40 + N0)
    pos = synth.poisson_particles(d, box, 2.0, 41)
    A = oracle.AMR(pos, N0, box, lmax, thr)
    keys, exists = _brute_structure(pos, N0, box, lmax, thr, want_exists=True)
    assert A.nlev == len(keys)
    for l in range(1, A.nlev):
        np.testing.assert_array_equal(A.keys(l), keys[l])
    # each particle's leaf level (the cube side of the adaptive CIC)
    lev = _brute_leaf_levels(pos, N0, box, exists)
    assert (lev > 0).any()
    np.testing.assert_array_equal(A.particle_levels(), lev)
    for l in range(A.nlev):
        assert A.counts(l).max() >= 0
    # every leaf holds at most thr particles unless it sits on the deepest level
    for l in range(A.nlev - 1 if A.nlev - 1 == lmax else A.nlev):
        leaf = A.refined(l) == 0
        if leaf.any():
            assert A.counts(l)[leaf].max() <= thr


# --------------------------------------------------------------------------
# Adaptive CIC (Sec. 3.1): brute force over the finest grid.  Every
# finest-level cell belongs to exactly one leaf (its deepest existing
# ancestor); the cube's overlap with each finest cell is a product of 1D
# overlaps; summing those per leaf gives the leaf masses.
# --------------------------------------------------------------------------
def test_adaptive_cic_brute_force():
    N0, box, lmax = 8, 8.0, 2
    rng = np.random.default_rng(3)
    clump = 2.3 + 0.6 * rng.random((150, 3))
    near = 1.05 + 0.4 * rng.random((6, 3))  # refined base cell, unrefined level-1 cell
    pos = np.concatenate([clump, near, box * rng.random((40, 3))])
    A = oracle.AMR(pos, N0, box, lmax, 8)
    assert A.nlev == 3
    A.deposit()
    Lf = A.nlev - 1
    Nf = N0 << Lf
    # leaf id of every finest cell: (level, cell index) via the oracle's keys
    leaf_of = {}
    keys = {l: A.keys(l) for l in range(1, A.nlev)}
    ref = {l: A.refined(l) for l in range(A.nlev)}

    def cell_index(l, I, J, K):
        Nl = N0 << l
        I, J, K = I % Nl, J % Nl, K % Nl
        if l == 0:
            return (I * Nl + J) * Nl + K
        Np_ = Nl // 2
        key = ((I // 2) * Np_ + J // 2) * Np_ + K // 2
        o = np.searchsorted(keys[l], key)
        if o >= len(keys[l]) or keys[l][o] != key:
            return -1
        return 8 * o + 4 * (I % 2) + 2 * (J % 2) + (K % 2)

    def leaf(I, J, K):
        for l in range(Lf, -1, -1):
            s = Lf - l
            c = cell_index(l, I >> s, J >> s, K >> s)
            if c >= 0:
                return l, c
        raise AssertionError

    mass = {l: np.zeros(A.ncell(l)) for l in range(A.nlev)}
    t = pos * (N0 / box)
    # cube sides from the brute-force structure, not from the oracle
    _, exists = _brute_structure(pos, N0, box, lmax, 8, want_exists=True)
    lev = _brute_leaf_levels(pos, N0, box, exists)
    np.testing.assert_array_equal(A.particle_levels(), lev)
    assert set(np.unique(lev)) == {0, 1, 2}
    for p in range(len(pos)):
        side = 2.0 ** -lev[p]
        lo = t[p] - side / 2
        hi = t[p] + side / 2
        rngs = [range(int(np.floor(lo[a] * 2 ** Lf)), int(np.floor(hi[a] * 2 ** Lf)) + 1) for a in range(3)]
        for I in rngs[0]:
            for J in rngs[1]:
                for K in rngs[2]:
                    ov = 1.0
                    for a, Q in enumerate((I, J, K)):
                        c0, c1 = Q * 2.0 ** -Lf, (Q + 1) * 2.0 ** -Lf
                        ov *= max(0.0, min(hi[a], c1) - max(lo[a], c0))
                    if ov > 0:
                        l, c = leaf(I, J, K)
                        mass[l][c] += ov / side ** 3
    for l in range(A.nlev):
        m = A.masses(l)
        leafmask = ref[l] == 0
        np.testing.assert_allclose(m[leafmask], mass[l][leafmask], rtol=0, atol=1e-12)
    assert abs(A.masses(0).sum() - len(pos)) < 1e-9


def test_uniform_cic_matches_standard_cic():
    """With no refinement the adaptive CIC is the textbook CIC."""
    N0, box = 16, 50.0
    rng = np.random.default_rng(8)
    pos = box * rng.random((500, 3))
    A = oracle.AMR(pos, N0, box, 0, 8)
    A.deposit()
    t = pos * (N0 / box) - 0.5
    i0 = np.floor(t).astype(int)
    w1 = t - i0
    ref = np.zeros((N0,) * 3)
    for a in (0, 1):
        for b in (0, 1):
            for c in (0, 1):
                w = (w1[:, 0] if a else 1 - w1[:, 0]) * (w1[:, 1] if b else 1 - w1[:, 1]) * \
                    (w1[:, 2] if c else 1 - w1[:, 2])
                np.add.at(ref, ((i0[:, 0] + a) % N0, (i0[:, 1] + b) % N0, (i0[:, 2] + c) % N0), w)
    np.testing.assert_allclose(A.masses(0).reshape(ref.shape), ref, atol=1e-12)


# --------------------------------------------------------------------------
# Ghosts (Sec. 3.3): linear reconstruction from the parent is exact for a
# field linear in space wherever both parent neighbours exist.
# --------------------------------------------------------------------------
def test_ghost_linear_reconstruction_exact_for_linear_field():
    N0, box = 16, 16.0
    rng = np.random.default_rng(4)
    pos = np.concatenate([6.0 + 3.0 * rng.random((400, 3))])
    A = oracle.AMR(pos, N0, box, 1, 8)
    assert A.nlev == 2
    x0 = (np.arange(N0) + 0.5)
    X, Y, Z = np.meshgrid(x0, x0, x0, indexing="ij")
    lin = lambda x, y, z: 0.3 * x - 0.2 * y + 0.1 * z + 1.0
    A.set_u(0, lin(X, Y, Z).ravel())
    g = A.ghosts(1)
    keys = A.keys(1)
    dirs = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    checked = 0
    for o, key in enumerate(keys):
        pi, pj, pk = key // (N0 * N0), (key // N0) % N0, key % N0
        for ch in range(8):
            I, J, K = 2 * pi + (ch >> 2 & 1), 2 * pj + (ch >> 1 & 1), 2 * pk + (ch & 1)
            for d, (a, b, c) in enumerate(dirs):
                v = g[8 * o + ch, d]
                if np.isnan(v):
                    continue
                gi, gj, gk = I + a, J + b, K + c  # ghost position, level-1 units
                assert 2 <= gi < 2 * N0 - 2 and 2 <= gj < 2 * N0 - 2 and 2 <= gk < 2 * N0 - 2
                exact = lin((gi + 0.5) / 2, (gj + 0.5) / 2, (gk + 0.5) / 2)
                assert abs(v - exact) < 1e-12
                checked += 1
    assert checked > 0


def test_ghost_reconstruction_error_for_quadratic_field():
    """Central slopes: for u = a x^2 + b y^2 + c z^2 + (linear) in coarse-cell
    units, P + s (u+ - u-)/8 at the daughter centre P + s/4 misses u there by
    exactly -(a + b + c)/16 (each axis: (x+1)^2 - (x-1)^2 = 4x, and
    (x + s/4)^2 - x^2 - s x/2 = 1/16).  A one-sided slope, a wrong daughter
    offset or a wrong factor gives an error that depends on the side s."""
    N0, box = 16, 16.0
    rng = np.random.default_rng(5)
    pos = 6.0 + 3.0 * rng.random((400, 3))
    A = oracle.AMR(pos, N0, box, 1, 8)
    assert A.nlev == 2
    x0 = np.arange(N0) + 0.5
    X, Y, Z = np.meshgrid(x0, x0, x0, indexing="ij")
    qa, qb, qc = 0.03, -0.01, 0.02  # a + b + c != 0
    quad = lambda x, y, z: qa * x * x + qb * y * y + qc * z * z + 0.3 * x - 0.1 * z + 1.0
    A.set_u(0, quad(X, Y, Z).ravel())
    g = A.ghosts(1)
    keys = A.keys(1)
    dirs = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    want = -(qa + qb + qc) / 16.0
    checked = 0
    for o, key in enumerate(keys):
        pi, pj, pk = key // (N0 * N0), (key // N0) % N0, key % N0
        for ch in range(8):
            I, J, K = 2 * pi + (ch >> 2 & 1), 2 * pj + (ch >> 1 & 1), 2 * pk + (ch & 1)
            for d, (a, b, c) in enumerate(dirs):
                v = g[8 * o + ch, d]
                if np.isnan(v):
                    continue
                gi, gj, gk = I + a, J + b, K + c
                exact = quad((gi + 0.5) / 2, (gj + 0.5) / 2, (gk + 0.5) / 2)
                assert abs((v - exact) - want) < 1e-12
                checked += 1
    assert checked > 0


def test_ghost_gradient_component_zero_where_parent_neighbour_missing():
    """Level-2 ghosts whose parent (a level-1 cell) lacks a level-1
    neighbour along an axis take that gradient component as 0 (Sec. 3.3,
    ghost cells from the parent by the linear reconstruction; reading: the
    component is dropped where one of the two neighbours does not exist).
    For a field linear in space, g . x, the reconstruction is exact along
    axes with both neighbours; along a dropped axis the ghost misses the
    exact value by -s g_d / 8 (base-cell units; daughter offset s/4 of a
    level-1 cell of side 1/2).  A tight clump just above a base-cell corner
    makes level 2 reach the edge of level 1."""
    N0, box = 8, 8.0
    rng = np.random.default_rng(11)
    pos = 3.02 + 0.05 * rng.random((60, 3))
    A = oracle.AMR(pos, N0, box, 2, 8)
    assert A.nlev == 3
    gvec = np.array([0.3, -0.2, 0.1])
    lin = lambda x, y, z: gvec[0] * x + gvec[1] * y + gvec[2] * z + 1.0
    x0 = np.arange(N0) + 0.5
    X, Y, Z = np.meshgrid(x0, x0, x0, indexing="ij")
    A.set_u(0, lin(X, Y, Z).ravel())
    keys1 = A.keys(1)
    kp = np.stack([keys1 // (N0 * N0), (keys1 // N0) % N0, keys1 % N0], 1)
    ch = np.array([[c >> 2 & 1, c >> 1 & 1, c & 1] for c in range(8)])
    cen1 = ((2 * kp[:, None, :] + ch[None, :, :]) + 0.5) / 2.0  # level-1 centres, base units
    A.set_u(1, lin(cen1[..., 0], cen1[..., 1], cen1[..., 2]).ravel())
    key1_set = set(int(k) for k in keys1)

    def exists1(I, J, K):  # level-1 cell exists iff its base parent is refined
        I, J, K = I % (2 * N0), J % (2 * N0), K % (2 * N0)
        return ((I // 2) * N0 + J // 2) * N0 + K // 2 in key1_set

    g = A.ghosts(2)
    keys2 = A.keys(2)
    N1 = 2 * N0
    dirs = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    n_drop = n_full = 0
    for o, key in enumerate(keys2):
        pi, pj, pk = key // (N1 * N1), (key // N1) % N1, key % N1
        for c in range(8):
            I, J, K = 2 * pi + (c >> 2 & 1), 2 * pj + (c >> 1 & 1), 2 * pk + (c & 1)
            for d, (a, b, cc) in enumerate(dirs):
                v = g[8 * o + c, d]
                if np.isnan(v):
                    continue
                G = np.array([I + a, J + b, K + cc])  # ghost, level-2 units
                P = G // 2                            # its parent, level-1 units
                assert exists1(*P)
                s = 2 * (G % 2) - 1                   # side of the ghost in its parent
                want = lin(*((G + 0.5) / 4.0))
                dropped = False
                for ax in range(3):
                    e = np.eye(3, dtype=np.int64)[ax]
                    if not (exists1(*(P + e)) and exists1(*(P - e))):
                        want -= s[ax] * gvec[ax] / 8.0
                        dropped = True
                assert abs(v - want) < 1e-12, (o, c, d, v, want)
                n_drop += dropped
                n_full += not dropped
    assert n_drop > 0 and n_full > 0, (n_drop, n_full)


# --------------------------------------------------------------------------
# P8: refining the whole box makes level 1 a uniform (2N)^3 grid with no
# patch boundary; its one-way solution must equal the uniform fine solve.
# --------------------------------------------------------------------------
def test_full_refinement_equals_uniform_fine_solve():
    N0, box, fr0 = 8, 50.0, 1e-5
    d = synth.lognormal_delta(2 * N0, box, 1.0, 50)
    pos = synth.poisson_particles(d, box, 4.0, 51)
    A = oracle.AMR(pos, N0, box, 1, -1)
    assert A.nlev == 2 and A.noct(1) == N0 ** 3
    A.deposit()
    A.set_model(fr0)
    rc, _ = A.solve(tol=1e-12)
    assert rc == 0
    # uniform (2N)^3 CIC of the same particles, solved by the dense solver
    B = oracle.AMR(pos, 2 * N0, box, 0, 8)
    B.deposit()
    dfine = B.delta(0).reshape((2 * N0,) * 3)
    uf, st = oracle.solve_dense(dfine, box, fr0, tol=1e-12)
    # map level-1 oct order (parent key, child 4a+2b+c) to dense (2N)^3
    u1 = A.u(1).reshape(-1, 2, 2, 2)
    keys = A.keys(1)
    pi, pj, pk = keys // (N0 * N0), (keys // N0) % N0, keys % N0
    dense = np.empty((2 * N0,) * 3)
    for a in (0, 1):
        for b in (0, 1):
            for c in (0, 1):
                dense[2 * pi + a, 2 * pj + b, 2 * pk + c] = u1[:, a, b, c]
    assert np.abs(dense - uf).max() < 1e-9
    # and level-1 delta equals the uniform CIC delta
    d1 = A.delta(1).reshape(-1, 2, 2, 2)
    dd = np.empty_like(dense)
    for a in (0, 1):
        for b in (0, 1):
            for c in (0, 1):
                dd[2 * pi + a, 2 * pj + b, 2 * pk + c] = d1[:, a, b, c]
    assert np.abs(dd - dfine).max() < 1e-10


def test_mass_conserved_on_every_level():
    N0, box = 16, 100.0
    d = synth.lognormal_delta(N0, box, 2.0, 60)
    pos = synth.poisson_particles(d, box, 3.0, 61)
    A = oracle.AMR(pos, N0, box, 3, 8)
    A.deposit()
    total = len(pos)
    leaf_sum = sum(A.masses(l)[A.refined(l) == 0].sum() for l in range(A.nlev))
    assert abs(leaf_sum - total) < 1e-9 * total
    assert abs(A.masses(0).sum() - total) < 1e-9 * total
    for l in range(1, A.nlev):
        # parents' mass equals the sum over their 8 daughters
        m = A.masses(l).reshape(-1, 8).sum(1)
        keys = A.keys(l)
        mp = A.masses(l - 1)
        if l == 1:
            np.testing.assert_allclose(mp[keys], m, rtol=1e-12, atol=1e-12)


def test_refined_level_one_way_manufactured():
    """Refined level with ghosts: f := L(u*) with the ghost values that the
    level's parent fixes; the level solve must return u* (unique solution)."""
    N0, box, fr0 = 16, 100.0, 1e-5
    d = synth.lognormal_delta(N0, box, 1.5, 70)
    pos = synth.poisson_particles(d, box, 1.0, 71)
    A = oracle.AMR(pos, N0, box, 1, 8)
    assert A.nlev == 2
    A.deposit()
    A.set_model(fr0)
    rng = np.random.default_rng(1)
    A.set_u(0, 0.2 * rng.standard_normal(A.ncell(0)))
    ustar = 0.3 * rng.standard_normal(A.ncell(1))
    A.set_u(1, ustar)
    A.set_source(1, np.zeros(A.ncell(1)))
    f = -A.residual(1)  # r = 0 - L(u*)  ->  f = L(u*)
    A.set_source(1, f)
    A.set_u(1, np.zeros(A.ncell(1)))
    rc, st = A.solve_level(1, tol=1e-12, init_from_parent=True)
    assert rc == 0
    assert np.abs(A.u(1) - ustar).max() < 1e-9


# --------------------------------------------------------------------------
# Force at the particles: with no refinement it is the textbook CIC
# interpolation of the grid force; with refinement the gather is the adjoint
# of the deposit, so sum_p acc_p = sum_leaves mass_leaf * acc_leaf.
# --------------------------------------------------------------------------
def test_particle_force_uniform_is_cic_interpolation():
    N0, box, fr0 = 16, 50.0, 1e-5
    d = synth.lognormal_delta(N0, box, 1.0, 80)
    pos = synth.poisson_particles(d, box, 1.0, 81)
    A = oracle.AMR(pos, N0, box, 0, 8)
    A.deposit()
    A.set_model(fr0)
    A.solve(tol=1e-10)
    fr, acc = oracle.force_dense(A.u(0).reshape((N0,) * 3), box, fr0)
    t = pos * (N0 / box) - 0.5
    i0 = np.floor(t).astype(int)
    w1 = t - i0
    ref = np.zeros((len(pos), 3))
    for a in (0, 1):
        for b in (0, 1):
            for c in (0, 1):
                w = (w1[:, 0] if a else 1 - w1[:, 0]) * (w1[:, 1] if b else 1 - w1[:, 1]) * \
                    (w1[:, 2] if c else 1 - w1[:, 2])
                ii = ((i0[:, 0] + a) % N0, (i0[:, 1] + b) % N0, (i0[:, 2] + c) % N0)
                for ax in range(3):
                    ref[:, ax] += w * acc[ax][ii]
    got = A.particle_force()
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_particle_force_is_adjoint_of_deposit():
    N0, box, fr0 = 16, 100.0, 1e-5
    d = synth.lognormal_delta(N0, box, 1.8, 90)
    pos = synth.poisson_particles(d, box, 2.0, 91)
    A = oracle.AMR(pos, N0, box, 2, 8)
    assert A.nlev == 3
    A.deposit()
    A.set_model(fr0)
    rc, _ = A.solve(tol=1e-9)
    assert rc == 0
    lhs = A.particle_force().sum(0)
    rhs = np.zeros(3)
    for l in range(A.nlev):
        leaf = A.refined(l) == 0
        _, acc = A.level_force(l)
        rhs += (A.masses(l)[leaf, None] * acc[leaf]).sum(0)
    assert np.abs(lhs - rhs).max() < 1e-10 * np.abs(A.particle_force()).sum()
