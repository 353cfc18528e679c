"""ctypes front end of the C oracle (``mgfr_oracle.c``).

TEST INFRASTRUCTURE ONLY: the CUDA product path never imports this module.
It compiles the oracle with gcc on first use (``build()``), in FP64 without
floating-point contraction, and exposes numpy-level helpers.  Every function
states the paper passage it follows; the arithmetic lives in the C file, but
for the periodic Poisson solve (numpy FFT).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mgfr_oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-fopenmp"]


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to its source (in-tree, git-ignored)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            d, i, ll, vp = C.c_double, C.c_int, C.c_longlong, C.c_void_p
            P = C.POINTER
            sig = {
                "orc_set_threads": (i, [i]),
                "orc_model_constants": (None, [d, d, i, d, vp]),
                "orc_effective_density": (None, [ll, vp, vp, d, d, i, d, vp]),
                "orc_amr_effective_pm": (None, [vp, i, vp]),
                "orc_amr_density_pm": (None, [vp, i, i, vp]),
                "orc_solve_dense": (i, [i, d, vp, d, d, i, d, vp, d, i, i, i, i, d, vp]),
                "orc_solve_dense_f": (i, [i, d, vp, d, d, i, d, vp, d, i, i, i, i, d, vp]),
                "orc_residual_dense": (None, [i, d, vp, d, d, i, d, vp, vp]),
                "orc_apply_L_dense": (None, [i, d, d, d, i, d, vp, vp]),
                "orc_residual_dense_at": (None, [i, d, d, d, i, d, vp, vp, vp, ll, vp]),
                "orc_force_dense": (None, [i, d, d, d, i, d, vp, vp, vp]),
                "orc_amr_create": (vp, [vp, ll, i, d, i, i]),
                "orc_amr_free": (None, [vp]),
                "orc_amr_nlev": (i, [vp]),
                "orc_amr_ncell": (ll, [vp, i]),
                "orc_amr_noct": (ll, [vp, i]),
                "orc_amr_keys": (None, [vp, i, vp]),
                "orc_amr_counts": (None, [vp, i, vp]),
                "orc_amr_refined": (None, [vp, i, vp]),
                "orc_amr_deposit": (None, [vp]),
                "orc_amr_masses": (None, [vp, i, vp]),
                "orc_amr_delta": (None, [vp, i, vp]),
                "orc_amr_set_model": (None, [vp, d, d, i, d]),
                "orc_amr_set_source": (None, [vp, i, vp]),
                "orc_amr_get_source": (None, [vp, i, vp]),
                "orc_amr_set_u": (None, [vp, i, vp]),
                "orc_amr_get_u": (None, [vp, i, vp]),
                "orc_amr_ghosts": (None, [vp, i, i, vp]),
                "orc_amr_residual": (d, [vp, i, i, vp]),
                "orc_amr_residual_at": (None, [vp, i, i, vp, ll, vp]),
                "orc_amr_solve_level": (i, [vp, i, d, ll, i, d, i, vp]),
                "orc_amr_solve": (i, [vp, d, i, ll, i, i, i, d, vp, vp]),
                "orc_amr_level_force": (None, [vp, i, i, vp, vp]),
                "orc_amr_particle_force": (None, [vp, i, vp]),
                "orc_amr_particle_levels": (None, [vp, vp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            L.orc_set_threads(1)  # one thread unless set_threads asks for more
            _lib = L
    return _lib


def set_threads(n: int) -> int:
    """Threads of the oracle's parallel loops (<= 0: all cores; 1 after
    loading); results do not depend on it.  Returns the number in use."""
    return int(lib().orc_set_threads(int(n)))


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# Default cosmology of the synthetic workloads: flat, Om = 0.3, n = 1.
OMEGA_M = 0.3


def model_constants(fr0_abs: float, a: float = 1.0, n: int = 1, omega_m: float = OMEGA_M) -> dict:
    """R~(a), fR_bar(a), alpha(a) and the source factor (Sec. 2, Eq. (10))."""
    out = np.zeros(4)
    lib().orc_model_constants(omega_m, fr0_abs, n, a, _p(out))
    return {"Rt": out[0], "fbar": out[1], "alpha": out[2], "src": out[3]}


def effective_density(u, delta, fr0_abs: float, a: float = 1.0, n: int = 1,
                      omega_m: float = OMEGA_M) -> np.ndarray:
    """delta rho_eff / rho_bar per cell from u and delta (Sec. 2.4, Eq.
    (31) with delta R from Eq. (11)); any level, any shape."""
    u = _f64(u)
    d = _f64(delta)
    assert u.shape == d.shape
    out = np.empty_like(u)
    lib().orc_effective_density(u.size, _p(u), _p(d), omega_m, fr0_abs, n, a, _p(out))
    return out


def poisson_periodic(rhs, box: float) -> np.ndarray:
    """phi with lap_h phi = rhs - mean(rhs) on a periodic N^3 grid, mean(phi) = 0,
    lap_h the 7-point Laplacian (spacing box/N): the exact solution of the
    discrete problem by FFT (the library transform is a step; the eigenvalues
    of lap_h are (2 cos(2 pi m / N) - 2) / h^2 per axis).  For the potential of
    the effective mass (Sec. 2.4, Eq. (30))."""
    r = _f64(rhs)
    N = r.shape[0]
    h = box / N
    m = np.arange(N)
    lam1 = (2.0 * np.cos(2.0 * np.pi * m / N) - 2.0) / (h * h)
    lamz = lam1[: N // 2 + 1]
    lam = lam1[:, None, None] + lam1[None, :, None] + lamz[None, None, :]
    rk = np.fft.rfftn(r)
    lam[0, 0, 0] = 1.0
    pk = rk / lam
    pk[0, 0, 0] = 0.0
    return np.fft.irfftn(pk, s=r.shape, axes=(0, 1, 2))


def pm_accel(phi, box: float, pos) -> np.ndarray:
    """-grad phi on a periodic N^3 grid by central differences at the cell
    centres, interpolated to the particles by cloud-in-cell (the 8 cells
    around x N / box - 1/2, product of the 1D linear weights): the PM force
    of Sec. 2.4.  phi (N, N, N), pos (Np, 3) in [0, box); returns (Np, 3)."""
    phi = _f64(phi)
    N = phi.shape[0]
    h = box / N
    g = [-(np.roll(phi, -1, ax) - np.roll(phi, 1, ax)) / (2.0 * h) for ax in range(3)]
    t = _f64(pos) / h - 0.5
    i0 = np.floor(t).astype(np.int64)
    w1 = t - i0
    acc = np.zeros((len(t), 3))
    for a in (0, 1):
        for b in (0, 1):
            for c in (0, 1):
                w = ((w1[:, 0] if a else 1.0 - w1[:, 0]) * (w1[:, 1] if b else 1.0 - w1[:, 1]) *
                     (w1[:, 2] if c else 1.0 - w1[:, 2]))
                I, J, K = (i0[:, 0] + a) % N, (i0[:, 1] + b) % N, (i0[:, 2] + c) % N
                for d in range(3):
                    acc[:, d] += w * g[d][I, J, K]
    return acc


def solve_dense(delta, box: float, fr0_abs: float, a: float = 1.0, n: int = 1,
                omega_m: float = OMEGA_M, u0=None, tol: float = 1e-8, max_vcycles: int = 100,
                n_pre: int = 2, n_post: int = 2, prolong_linear: bool = True,
                step_cap: float = 2.0, f=None):
    """FAS-multigrid NGS solve on a periodic N^3 grid (Sec. 3.3, steps 1-8).

    Returns (u, stats) with stats keys vcycles, res0, res, resmax, fnorm,
    updates, converged.  If ``f`` is given it replaces the source built from
    ``delta`` (manufactured right-hand sides).
    """
    delta = _f64(delta)
    N = delta.shape[0]
    u = np.zeros_like(delta) if u0 is None else _f64(u0).copy()
    st = np.zeros(8)
    if f is None:
        lib().orc_solve_dense(N, box, _p(delta), omega_m, fr0_abs, n, a, _p(u), tol, max_vcycles,
                              n_pre, n_post, int(prolong_linear), step_cap, _p(st))
    else:
        f = _f64(f)
        lib().orc_solve_dense_f(N, box, _p(f), omega_m, fr0_abs, n, a, _p(u), tol, max_vcycles,
                                n_pre, n_post, int(prolong_linear), step_cap, _p(st))
    keys = ["vcycles", "res0", "res", "resmax", "fnorm", "updates", "converged"]
    return u, {k: float(st[i]) for i, k in enumerate(keys)}


def residual_dense(u, delta, box, fr0_abs, a=1.0, n=1, omega_m=OMEGA_M):
    """r = f - L(u) on a dense periodic grid (Sec. 3.2)."""
    u, delta = _f64(u), _f64(delta)
    r = np.empty_like(u)
    lib().orc_residual_dense(u.shape[0], box, _p(delta), omega_m, fr0_abs, n, a, _p(u), _p(r))
    return r


def apply_L_dense(u, box, fr0_abs, a=1.0, n=1, omega_m=OMEGA_M):
    """L(u) on a dense periodic grid (Sec. 3.2)."""
    u = _f64(u)
    out = np.empty_like(u)
    lib().orc_apply_L_dense(u.shape[0], box, omega_m, fr0_abs, n, a, _p(u), _p(out))
    return out


def residual_dense_at(u, delta, cells, box, fr0_abs, a=1.0, n=1, omega_m=OMEGA_M):
    """r = f - L(u) at the given linear cell indices only."""
    u, delta = _f64(u), _f64(delta)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    r = np.empty(len(cells))
    lib().orc_residual_dense_at(u.shape[0], box, omega_m, fr0_abs, n, a, _p(u), _p(delta),
                                _p(cells), len(cells), _p(r))
    return r


def force_dense(u, box, fr0_abs, a=1.0, n=1, omega_m=OMEGA_M):
    """fR = fR_bar e^u and a_MG/c^2 = grad fR / (2a) [3,N,N,N] (Sec. 2)."""
    u = _f64(u)
    N = u.shape[0]
    fr = np.empty_like(u)
    acc = np.empty((3,) + u.shape)
    lib().orc_force_dense(N, box, omega_m, fr0_abs, n, a, _p(u), _p(fr), _p(acc))
    return fr, acc


class AMR:
    """Refinement hierarchy, adaptive CIC and one-way level solves (Sec. 3.1, 3.3)."""

    def __init__(self, pos, N0: int, box: float, lmax: int, refine_count: int = 8):
        self.pos = _f64(pos).reshape(-1, 3)
        self.N0, self.box = N0, box
        self.h = lib().orc_amr_create(_p(self.pos), len(self.pos), N0, box, lmax, refine_count)
        self.model = None

    def close(self):
        if self.h:
            lib().orc_amr_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nlev(self) -> int:
        return lib().orc_amr_nlev(self.h)

    def ncell(self, l):
        return lib().orc_amr_ncell(self.h, l)

    def noct(self, l):
        return lib().orc_amr_noct(self.h, l)

    def keys(self, l):
        out = np.empty(self.noct(l), dtype=np.int64)
        lib().orc_amr_keys(self.h, l, _p(out))
        return out

    def counts(self, l):
        out = np.empty(self.ncell(l), dtype=np.int32)
        lib().orc_amr_counts(self.h, l, _p(out))
        return out

    def refined(self, l):
        out = np.empty(self.ncell(l), dtype=np.uint8)
        lib().orc_amr_refined(self.h, l, _p(out))
        return out

    def deposit(self):
        lib().orc_amr_deposit(self.h)

    def masses(self, l):
        out = np.empty(self.ncell(l))
        lib().orc_amr_masses(self.h, l, _p(out))
        return out

    def delta(self, l):
        out = np.empty(self.ncell(l))
        lib().orc_amr_delta(self.h, l, _p(out))
        return out

    def set_model(self, fr0_abs, a=1.0, n=1, omega_m=OMEGA_M):
        self.model = (fr0_abs, a, n, omega_m)
        lib().orc_amr_set_model(self.h, omega_m, fr0_abs, n, a)

    def set_source(self, l, f):
        lib().orc_amr_set_source(self.h, l, _p(_f64(f)))

    def source(self, l):
        out = np.empty(self.ncell(l))
        lib().orc_amr_get_source(self.h, l, _p(out))
        return out

    def set_u(self, l, u):
        lib().orc_amr_set_u(self.h, l, _p(_f64(u)))

    def u(self, l):
        out = np.empty(self.ncell(l))
        lib().orc_amr_get_u(self.h, l, _p(out))
        return out

    def ghosts(self, l, prolong_linear=True):
        out = np.empty(6 * self.ncell(l))
        lib().orc_amr_ghosts(self.h, l, int(prolong_linear), _p(out))
        return out.reshape(-1, 6)

    def residual(self, l, prolong_linear=True):
        r = np.empty(self.ncell(l))
        lib().orc_amr_residual(self.h, l, int(prolong_linear), _p(r))
        return r

    def residual_at(self, l, cells, prolong_linear=True):
        """f - L(u) at the given cells of level l (current u of levels l, l-1)."""
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        r = np.empty(len(cells))
        lib().orc_amr_residual_at(self.h, l, int(prolong_linear), _p(cells), len(cells), _p(r))
        return r

    def solve_level(self, l, tol=1e-8, max_sweeps=200000, prolong_linear=True, step_cap=2.0,
                    init_from_parent=True):
        out = np.zeros(4)
        rc = lib().orc_amr_solve_level(self.h, l, tol, max_sweeps, int(prolong_linear), step_cap,
                                       int(init_from_parent), _p(out))
        return rc, {"sweeps": out[0], "res0": out[1], "res": out[2], "fnorm": out[3]}

    def solve(self, tol=1e-8, max_vcycles=100, max_sweeps_refined=200000, n_pre=2, n_post=2,
              prolong_linear=True, step_cap=2.0, u0_base=None):
        """One-way solve of every level (Sec. 3.3, steps 1-12)."""
        st = np.zeros(4 + 4 * 16)
        u0 = None if u0_base is None else _f64(u0_base)
        rc = lib().orc_amr_solve(self.h, tol, max_vcycles, max_sweeps_refined, n_pre, n_post,
                                 int(prolong_linear), step_cap, _p(u0), _p(st))
        return rc, st

    def effective_pm(self, lpm: int = 0) -> np.ndarray:
        """Effective mass density contrast of the solved hierarchy on the
        periodic PM grid of level lpm (Sec. 2.4: each leaf cell's effective
        mass shared among the PM cells it overlaps by volume)."""
        Npm = self.N0 << lpm
        out = np.empty((Npm, Npm, Npm))
        lib().orc_amr_effective_pm(self.h, lpm, _p(out))
        return out

    def density_pm(self, lpm: int = 0, what: int = 2) -> np.ndarray:
        """Density contrast on the periodic PM grid of level lpm, each leaf
        cell's share by overlapping volume (Sec. 2.4): what 0 the effective
        mass, 1 the matter, 2 both (the right-hand side of Eq. (30))."""
        Npm = self.N0 << lpm
        out = np.empty((Npm, Npm, Npm))
        lib().orc_amr_density_pm(self.h, lpm, what, _p(out))
        return out

    def pm_potential(self, lpm: int = 0, what: int = 2) -> np.ndarray:
        """Comoving potential on the PM grid of level lpm (Sec. 2.4, Eq. (30)):
        lap_x phi = 4 pi G a^2 rho_bar (delta_pm - mean) = (3/2) Om H0^2 a^-1
        (delta_pm - mean), with H0 = 100 km/s per Mpc/h, so phi is in (km/s)^2
        and x in Mpc/h; the 7-point periodic problem solved exactly by FFT,
        mean(phi) = 0."""
        fr0, a, n, om = self.model
        rhs = 1.5e4 * om / a * self.density_pm(lpm, what)
        return poisson_periodic(rhs, self.box)

    def level_force(self, l, prolong_linear=True):
        n = self.ncell(l)
        fr = np.empty(n)
        acc = np.empty((n, 3))
        lib().orc_amr_level_force(self.h, l, int(prolong_linear), _p(fr), _p(acc))
        return fr, acc

    def particle_force(self, prolong_linear=True):
        acc = np.empty((len(self.pos), 3))
        lib().orc_amr_particle_force(self.h, int(prolong_linear), _p(acc))
        return acc

    def particle_levels(self):
        out = np.empty(len(self.pos), dtype=np.int32)
        lib().orc_amr_particle_levels(self.h, _p(out))
        return out
