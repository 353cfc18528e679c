"""Thin ctypes binding of libmgfr.so (the C ABI declared in include/mgfr.h).

Argument marshalling only: every step of the solve runs in the library's CUDA
kernels.  Inputs and outputs are torch CUDA tensors (FP64, contiguous); a
Solver's work is ordered after the stream it was created on (torch's current
stream at that time, unless one is passed).  There is no CPU fallback: if the
library is missing, loading it raises.
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libmgfr.so")

MGFR_OK, MGFR_E_INVALID, MGFR_E_CUDA, MGFR_E_OOM, MGFR_E_NOCONVERGE, MGFR_E_TIMEOUT, \
    MGFR_E_UNSUPPORTED = range(7)
STATUS_NAMES = ["OK", "INVALID", "CUDA", "OOM", "NOCONVERGE", "TIMEOUT", "UNSUPPORTED"]
PREC_FP64, PREC_MIXED = 0, 1
START_ZERO, START_USER, START_LEARNED, START_PREVIOUS, START_PREVIOUS_ALL = 0, 1, 2, 3, 4
PM_EFFECTIVE, PM_MATTER, PM_TOTAL = 0, 1, 2
FIELD_U, FIELD_FR, FIELD_SOURCE, FIELD_MASS, FIELD_ACC, FIELD_COUNT = range(6)


class Config(C.Structure):
    _fields_ = [
        ("omega_m", C.c_double), ("fr0_abs", C.c_double), ("n", C.c_int),
        ("precision", C.c_int), ("tol_rel", C.c_double), ("n_pre", C.c_int),
        ("n_post", C.c_int), ("max_vcycles", C.c_int), ("prolong_linear", C.c_int),
        ("step_cap", C.c_double), ("max_level", C.c_int), ("refine_count", C.c_int),
        ("mixed_switch", C.c_double), ("mixed_inner", C.c_int), ("max_spins", C.c_longlong),
        ("profile", C.c_int), ("mask_thres", C.c_double), ("n_coarse", C.c_int),
        ("start", C.c_int),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("vcycles", C.c_int), ("outer_iters", C.c_int), ("cell_updates", C.c_longlong),
        ("linear_updates", C.c_longlong), ("res_l2_init", C.c_double),
        ("res_l2_final", C.c_double), ("res_max_final", C.c_double), ("f_l2", C.c_double),
        ("t_total_ms", C.c_double), ("t_solve_ms", C.c_double), ("n_levels", C.c_int),
        ("cells_per_level", C.c_longlong * 16), ("octs_per_level", C.c_longlong * 16),
        ("level_iters", C.c_int * 16), ("level_res", C.c_double * 16),
        ("kern_ms", C.c_double * 6), ("kern_launches", C.c_longlong * 6),
        ("kern_cells", C.c_longlong * 6), ("gpu_launches", C.c_longlong),
    ]

    def to_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if hasattr(v, "__len__") else v
        return out


class BatchItem(C.Structure):
    _fields_ = [
        ("N", C.c_int), ("box", C.c_double), ("a", C.c_double), ("fr0_abs", C.c_double),
        ("n", C.c_int), ("delta_dev", C.c_void_p), ("u_init_dev", C.c_void_p),
        ("fr_out_dev", C.c_void_p), ("acc_out_dev", C.c_void_p), ("u_out_dev", C.c_void_p),
    ]


class MGFRError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"mgfr {STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


_lib = None

# name -> (restype, argtypes); every symbol that include/mgfr.h declares.
SIGNATURES = {
    "mgfr_version": (C.c_char_p, []),
    "mgfr_config_default": (None, [C.c_void_p]),
    "mgfr_create": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "mgfr_set_config": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mgfr_solve_density": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_double,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p]),
    "mgfr_solve_particles": (C.c_int, [C.c_void_p, C.c_void_p, C.c_longlong, C.c_int, C.c_double,
                                       C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p]),
    "mgfr_solve_particles_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_longlong, C.c_int,
                                            C.c_double, C.c_double, C.c_void_p, C.c_void_p,
                                            C.c_void_p, C.c_void_p]),
    "mgfr_get_level_info": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "mgfr_get_level_keys": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "mgfr_get_level_field": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p]),
    "mgfr_get_effective_density": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "mgfr_effective_mass_pm": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "mgfr_pm_potential": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                    C.c_void_p]),
    "mgfr_pm_accel": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_longlong,
                                C.c_void_p, C.c_void_p]),
    "mgfr_kick_drift": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_longlong, C.c_double,
                                  C.c_double, C.c_double, C.c_void_p]),
    "mgfr_solve_density_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                                             C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.c_void_p]),
    "mgfr_batch_solve": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "mgfr_batch_autotune": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mgfr_unet_init": (C.c_int, [C.c_void_p, C.c_ulonglong]),
    "mgfr_unet_train_step": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_float, C.c_void_p]),
    "mgfr_unet_predict": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_double, C.c_void_p]),
    "mgfr_unet_params": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "mgfr_unet_grads": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mgfr_unet_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "mgfr_unet_load": (C.c_int, [C.c_void_p, C.c_char_p]),
    "mgfr_nn_conv3d": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p]),
    "mgfr_last_error": (C.c_char_p, [C.c_void_p]),
    "mgfr_destroy": (None, [C.c_void_p]),
}


def lib():
    """Load libmgfr.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_1305_2418_gb300.build")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def default_config(**kw) -> Config:
    cfg = Config()
    lib().mgfr_config_default(C.byref(cfg))
    for k, v in kw.items():
        if not hasattr(cfg, k):
            raise KeyError(k)
        setattr(cfg, k, v)
    return cfg


def _ptr(t):
    if t is None:
        return None
    import torch
    assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous(), "need contiguous CUDA FP64"
    return C.c_void_p(t.data_ptr())


class Solver:
    """A library context bound to one device and one stream (torch's current
    stream when the Solver is created, unless `stream` is given)."""

    def __init__(self, device: int = 0, stream=None, **cfg):
        import torch
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        self.cfg = default_config(**cfg)
        h = C.c_void_p()
        st = lib().mgfr_create(C.byref(h), C.byref(self.cfg), device, C.c_void_p(stream.cuda_stream))
        if st != MGFR_OK:
            raise MGFRError(st, "mgfr_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().mgfr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return lib().mgfr_last_error(self.h).decode()

    def set_config(self, **kw):
        for k, v in kw.items():
            setattr(self.cfg, k, v)
        st = lib().mgfr_set_config(self.h, C.byref(self.cfg))
        if st != MGFR_OK:
            raise MGFRError(st, self.last_error())

    def _check(self, st, allow_noconverge=False):
        if st == MGFR_OK or (allow_noconverge and st == MGFR_E_NOCONVERGE):
            return st
        raise MGFRError(st, self.last_error())

    def solve_density(self, delta, box: float, a: float = 1.0, u_init=None, want_acc=True,
                      want_u=False, allow_noconverge=False):
        """f_R (and force, u) on a periodic N^3 grid from delta (mgfr_solve_density)."""
        import torch
        N = delta.shape[0]
        fr = torch.empty_like(delta)
        acc = torch.empty((3,) + tuple(delta.shape), dtype=delta.dtype, device=delta.device) \
            if want_acc else None
        u = torch.empty_like(delta) if want_u else None
        stats = Stats()
        st = lib().mgfr_solve_density(self.h, _ptr(delta), N, box, a, _ptr(u_init), _ptr(fr),
                                      _ptr(acc), _ptr(u), C.byref(stats))
        self._check(st, allow_noconverge)
        return {"fr": fr, "acc": acc, "u": u, "stats": stats.to_dict(), "status": st}

    def solve_particles(self, pos, N_base: int, box: float, a: float = 1.0, u_init=None,
                        want_fr=True, want_acc=True, allow_noconverge=False):
        """f_R on the base grid and the force at the particles (mgfr_solve_particles)."""
        import torch
        assert pos.ndim == 2 and pos.shape[1] == 3
        fr = torch.empty((N_base,) * 3, dtype=torch.float64, device=pos.device) if want_fr else None
        acc = torch.empty_like(pos) if want_acc else None
        stats = Stats()
        st = lib().mgfr_solve_particles(self.h, _ptr(pos), pos.shape[0], N_base, box, a,
                                        _ptr(u_init), _ptr(fr), _ptr(acc), C.byref(stats))
        self._check(st, allow_noconverge)
        return {"fr": fr, "acc": acc, "stats": stats.to_dict(), "status": st}

    def solve_particles_host(self, pos_host, N_base: int, box: float, a: float = 1.0,
                             acc_out=None, u_init=None, want_fr=False, allow_noconverge=False):
        """mgfr_solve_particles_host: positions and forces in host memory (CPU FP64
        tensors, contiguous; page-locked ones let the copies overlap the gather)."""
        import torch
        assert pos_host.device.type == "cpu" and pos_host.dtype == torch.float64
        assert pos_host.is_contiguous() and pos_host.ndim == 2 and pos_host.shape[1] == 3
        if acc_out is None:
            acc_out = torch.empty_like(pos_host, pin_memory=pos_host.is_pinned())
        assert acc_out.device.type == "cpu" and acc_out.dtype == torch.float64
        assert acc_out.is_contiguous() and acc_out.shape == pos_host.shape
        fr = torch.empty((N_base,) * 3, dtype=torch.float64, device=f"cuda:{self.device}") \
            if want_fr else None
        stats = Stats()
        st = lib().mgfr_solve_particles_host(
            self.h, C.c_void_p(pos_host.data_ptr()), pos_host.shape[0], N_base, box, a,
            _ptr(u_init), _ptr(fr), C.c_void_p(acc_out.data_ptr()), C.byref(stats))
        self._check(st, allow_noconverge)
        return {"fr": fr, "acc": acc_out, "stats": stats.to_dict(), "status": st}

    def level_info(self, level: int):
        no, nc = C.c_longlong(), C.c_longlong()
        self._check(lib().mgfr_get_level_info(self.h, level, C.byref(no), C.byref(nc)))
        return no.value, nc.value

    def level_keys(self, level: int):
        import numpy as np
        no, _ = self.level_info(level)
        out = np.empty(no, dtype=np.int64)
        self._check(lib().mgfr_get_level_keys(self.h, level, out.ctypes.data_as(C.c_void_p)))
        return out

    def level_field(self, level: int, what: int):
        import numpy as np
        _, nc = self.level_info(level)
        out = np.empty(3 * nc if what == FIELD_ACC else nc)
        self._check(lib().mgfr_get_level_field(self.h, level, what, out.ctypes.data_as(C.c_void_p)))
        return out

    def effective_density(self, level: int):
        """delta rho_eff / rho_bar per cell of a level of the last particle
        solve (mgfr_get_effective_density), as a CUDA FP64 tensor."""
        import torch
        _, nc = self.level_info(level)
        out = torch.empty(nc, dtype=torch.float64, device=f"cuda:{self.device}")
        self._check(lib().mgfr_get_effective_density(self.h, level, _ptr(out)))
        return out

    def effective_mass_pm(self, N_base: int, lpm: int = 0):
        """The effective mass on the periodic PM grid of level lpm
        (mgfr_effective_mass_pm), as a CUDA FP64 tensor of shape (N_pm,)*3."""
        import torch
        Npm = N_base << lpm
        out = torch.empty((Npm,) * 3, dtype=torch.float64, device=f"cuda:{self.device}")
        self._check(lib().mgfr_effective_mass_pm(self.h, lpm, _ptr(out)))
        return out

    def pm_potential(self, N_base: int, lpm: int = 0, what: int = 2, want_density=False):
        """Potential (km/s)^2 on the periodic PM grid of level lpm (mgfr_pm_potential):
        returns (phi, delta_pm or None, stats)."""
        import torch
        Npm = N_base << lpm
        phi = torch.empty((Npm,) * 3, dtype=torch.float64, device=f"cuda:{self.device}")
        dens = torch.empty_like(phi) if want_density else None
        stats = Stats()
        self._check(lib().mgfr_pm_potential(self.h, lpm, what, _ptr(phi), _ptr(dens),
                                            C.byref(stats)))
        return phi, dens, stats.to_dict()

    def pm_accel(self, pos, lpm: int = 0, what: int = 2):
        """-grad phi of the PM potential at the particles (mgfr_pm_accel):
        returns (acc [Np, 3] CUDA FP64, stats)."""
        acc = torch_empty_like(pos)
        stats = Stats()
        self._check(lib().mgfr_pm_accel(self.h, lpm, what, _ptr(pos), pos.shape[0], _ptr(acc),
                                        C.byref(stats)))
        return acc, stats.to_dict()

    def _batch_items(self, deltas, boxes, a, fr0s, ns, u_inits, want_acc, want_u=False):
        import torch
        k = len(deltas)
        items = (BatchItem * k)()
        outs = []
        for i, d in enumerate(deltas):
            fr = torch.empty_like(d)
            acc = torch.empty((3,) + tuple(d.shape), dtype=d.dtype, device=d.device) \
                if want_acc else None
            u = torch.empty_like(d) if want_u else None
            outs.append({"fr": fr, "acc": acc, "u": u})
            u0 = None if u_inits is None else u_inits[i]
            items[i] = BatchItem(d.shape[0], boxes[i], a[i], fr0s[i], ns[i], _ptr(d), _ptr(u0),
                                 _ptr(fr), _ptr(acc), _ptr(u))
        return items, outs

    def batch_solve(self, deltas, boxes, fr0s, a=None, ns=None, u_inits=None, want_acc=False,
                    want_u=False, allow_noconverge=False):
        """Many independent periodic solves in one persistent launch (mgfr_batch_solve)."""
        k = len(deltas)
        a = [1.0] * k if a is None else a
        ns = [1] * k if ns is None else ns
        items, outs = self._batch_items(deltas, boxes, a, fr0s, ns, u_inits, want_acc, want_u)
        stats = (Stats * k)()
        st = lib().mgfr_batch_solve(self.h, k, items, stats)
        self._check(st, allow_noconverge)
        for i in range(k):
            outs[i]["stats"] = stats[i].to_dict()
        return outs, st

    def batch_autotune(self, deltas, boxes, fr0s, a=None, ns=None):
        k = len(deltas)
        a = [1.0] * k if a is None else a
        ns = [1] * k if ns is None else ns
        items, _ = self._batch_items(deltas, boxes, a, fr0s, ns, None, False)
        t, b = C.c_int(), C.c_int()
        self._check(lib().mgfr_batch_autotune(self.h, k, items, C.byref(t), C.byref(b)), True)
        return t.value, b.value

    # ---- learned initial guess (U-Net) ----
    def unet_init(self, seed: int = 0):
        self._check(lib().mgfr_unet_init(self.h, seed))

    def unet_train_step(self, deltas, fr0s, targets, lr=1e-3):
        """One Adam step on a batch: deltas/targets [B, D, D, D] CUDA FP64."""
        import numpy as np
        B, D = deltas.shape[0], deltas.shape[1]
        fr = np.ascontiguousarray(fr0s, dtype=np.float64)
        loss = C.c_double()
        self._check(lib().mgfr_unet_train_step(self.h, B, D, _ptr(deltas.contiguous()),
                                               fr.ctypes.data_as(C.c_void_p),
                                               _ptr(targets.contiguous()), lr, C.byref(loss)))
        return loss.value

    def unet_predict(self, delta, fr0_abs):
        import torch
        u = torch.empty_like(delta)
        self._check(lib().mgfr_unet_predict(self.h, delta.shape[0], _ptr(delta), fr0_abs, _ptr(u)))
        return u

    def unet_params(self):
        import numpy as np
        n = C.c_longlong()
        self._check(lib().mgfr_unet_params(self.h, 0, None, C.byref(n)))
        out = np.empty(n.value, dtype=np.float32)
        self._check(lib().mgfr_unet_params(self.h, 0, out.ctypes.data_as(C.c_void_p), None))
        return out

    def unet_set_params(self, p):
        import numpy as np
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._check(lib().mgfr_unet_params(self.h, 1, p.ctypes.data_as(C.c_void_p), None))

    def unet_save(self, path: str):
        self._check(lib().mgfr_unet_save(self.h, os.fsencode(path)))

    def unet_load(self, path: str):
        self._check(lib().mgfr_unet_load(self.h, os.fsencode(path)))

    def unet_grads(self):
        import numpy as np
        n = C.c_longlong()
        self._check(lib().mgfr_unet_params(self.h, 0, None, C.byref(n)))
        out = np.empty(n.value, dtype=np.float32)
        self._check(lib().mgfr_unet_grads(self.h, out.ctypes.data_as(C.c_void_p)))
        return out


def torch_empty_like(t):
    import torch
    return torch.empty_like(t)


def kick_drift(pos, vel, acc, kick: float, drift: float, box: float, stream=None):
    """Leapfrog kick-drift of [Np, 3] CUDA FP64 arrays in place (mgfr_kick_drift)."""
    import torch
    s = torch.cuda.current_stream(pos.device) if stream is None else stream
    st = lib().mgfr_kick_drift(_ptr(pos), _ptr(vel), _ptr(acc), pos.shape[0], kick, drift, box,
                               C.c_void_p(s.cuda_stream))
    if st != MGFR_OK:
        raise MGFRError(st, "mgfr_kick_drift failed")


def conv3d(op, x, w, bias=None, relu=False, g=None, db=None, stream=None):
    """Convolution primitive of the network (mgfr_nn_conv3d) on torch tensors:
    x [B, D, D, D, Cin] bf16, w [27, Cin, Cout] bf16, g [B, D, D, D, Cout] bf16."""
    import torch
    B, D = x.shape[0], x.shape[1]
    Cin, Cout = w.shape[1], w.shape[2]
    if op == 0:
        out = torch.empty(x.shape[:-1] + (Cout,), dtype=torch.bfloat16, device=x.device)
    elif op == 1:
        out = torch.empty(x.shape, dtype=torch.float32, device=x.device)
    else:
        out = torch.empty((27, Cin, Cout), dtype=torch.float32, device=x.device)
    s = torch.cuda.current_stream(x.device) if stream is None else stream
    vp = lambda t: None if t is None else C.c_void_p(t.data_ptr())
    st = lib().mgfr_nn_conv3d(op, B, D, Cin, Cout, vp(x), vp(w), vp(bias), int(relu), vp(g),
                              vp(out), vp(db), C.c_void_p(s.cuda_stream))
    if st != MGFR_OK:
        raise MGFRError(st, "mgfr_nn_conv3d failed")
    return out
