"""ctypes binding of the C ABI in include/prop.h (argument marshalling only).

Every function keeps its C name and argument order; device buffers are passed
as integer addresses (``tensor.data_ptr()``), host buffers as numpy arrays.
The library must exist (``paper_2410_17446_gb300.build``): there is no
fallback, and loading fails loudly when it is missing.

``Propagator`` is a thin convenience wrapper that takes its workspace from
torch and its stream from ``torch.cuda.current_stream()``.
"""
from __future__ import annotations

import ctypes as ct
import os
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libprop.so")

(PROP_OK, PROP_E_ARG, PROP_E_WORKSPACE, PROP_E_CUDA, PROP_E_NOCONV, PROP_E_NAN, PROP_E_UNSUPPORTED, PROP_E_SCRATCH,
 PROP_E_TIMEOUT) = range(9)
PROP_FP64, PROP_FP32 = 0, 1


class prop_grid(ct.Structure):
    _fields_ = [("nx", ct.c_int32), ("ny", ct.c_int32), ("dx", ct.c_double), ("dy", ct.c_double)]


class prop_opts(ct.Structure):
    _fields_ = [("ncomp", ct.c_int32), ("precision", ct.c_int32), ("restart", ct.c_int32),
                ("max_restarts", ct.c_int32), ("tol", ct.c_double), ("guess", ct.c_int32),
                ("precond", ct.c_int32), ("form", ct.c_int32), ("substeps", ct.c_int32),
                ("multigroup", ct.c_int32)]


PROP_GUESS_ZERO, PROP_GUESS_LEARNED = 0, 1
PROP_ROWS_BLOCK, PROP_ROWS_WARP = 0, 1
PROP_COLS_TMA, PROP_COLS_PLAIN, PROP_COLS_WARP = 0, 1, 2


PROP_FFT_SMALL_ITEMS = 2


class prop_fft_plan(ct.Structure):
    _fields_ = [("rows", ct.c_int32), ("cols", ct.c_int32), ("rows_small", ct.c_int32), ("cols_small", ct.c_int32)]
PROP_PRECOND_FREESPACE, PROP_PRECOND_MEAN = 0, 1
PROP_FORM_EXPONENTIAL, PROP_FORM_PSEUDODIFF = 0, 1
PROP_GUESS_CHANNELS = 16


class prop_stats(ct.Structure):
    _fields_ = [("steps", ct.c_int64), ("npoles", ct.c_int32), ("nbeams", ct.c_int32),
                ("last_iters_max", ct.c_int32), ("last_cycles_max", ct.c_int32),
                ("last_iters_sum", ct.c_int64), ("last_resid_max", ct.c_double),
                ("total_iters", ct.c_int64), ("kernel_launches", ct.c_int64)]


PROP_NKINDS = 13


class prop_kernel_profile(ct.Structure):
    _fields_ = [("name", ct.c_char * 24), ("launches", ct.c_int64), ("total_ms", ct.c_double),
                ("alg_bytes", ct.c_double)]


MEDIUM_FN = ct.CFUNCTYPE(ct.c_int, ct.c_void_p, ct.c_int32, ct.c_void_p)

_lib = None

_SIGS = {
    "prop_default_opts": (ct.c_int, [ct.POINTER(prop_opts), ct.c_int32, ct.c_int32]),
    "prop_workspace_size": (ct.c_int, [ct.c_int32, ct.POINTER(prop_grid), ct.c_int32, ct.POINTER(prop_opts),
                                       ct.POINTER(ct.c_size_t)]),
    "prop_create": (ct.c_int, [ct.c_int32, ct.POINTER(prop_grid), ct.c_double, ct.c_double, ct.c_double,
                               ct.c_int32, ct.POINTER(ct.c_double), ct.POINTER(ct.c_double),
                               ct.POINTER(ct.c_double), ct.POINTER(prop_opts), ct.c_void_p, ct.c_size_t,
                               ct.c_void_p, ct.POINTER(ct.c_void_p)]),
    "prop_set_medium": (ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_void_p]),
    "prop_set_field": (ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_void_p]),
    "prop_get_field": (ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_void_p]),
    "prop_step": (ct.c_int, [ct.c_void_p]),
    "prop_get_substeps": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int32)]),
    "prop_get_fft_plan": (ct.c_int, [ct.c_int32, ct.c_int32, ct.POINTER(prop_fft_plan)]),
    "prop_set_fft_plan": (ct.c_int, [ct.c_int32, ct.c_int32, ct.POINTER(prop_fft_plan)]),
    "prop_fft_autotune_workspace_size": (ct.c_int, [ct.c_int32, ct.c_int32, ct.c_int32, ct.POINTER(ct.c_size_t)]),
    "prop_fft_autotune": (ct.c_int, [ct.c_int32, ct.c_int32, ct.c_int32, ct.c_int32, ct.c_int32, ct.c_void_p,
                                     ct.c_size_t, ct.c_void_p, ct.POINTER(prop_fft_plan), ct.POINTER(ct.c_float)]),
    "prop_get_e3": (ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_void_p]),
    "prop_run": (ct.c_int, [ct.c_void_p, ct.c_int32, MEDIUM_FN, ct.c_void_p]),
    "prop_get_stats": (ct.c_int, [ct.c_void_p, ct.POINTER(prop_stats)]),
    "prop_get_iterations": (ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int32)]),
    "prop_error_string": (ct.c_char_p, [ct.c_int]),
    "prop_set_profiling": (ct.c_int, [ct.c_void_p, ct.c_int32]),
    "prop_get_profile": (ct.c_int, [ct.c_void_p, ct.POINTER(prop_kernel_profile)]),
    "prop_destroy": (None, [ct.c_void_p]),
    "prop_fft2_workspace_size": (ct.c_int, [ct.c_int32, ct.c_int32, ct.c_int32, ct.POINTER(ct.c_size_t)]),
    "prop_fft2": (ct.c_int, [ct.c_int32, ct.c_int32, ct.c_int32, ct.c_int32, ct.c_int32, ct.c_void_p,
                             ct.c_void_p, ct.c_size_t, ct.c_void_p]),
    "prop_apply_freespace_inverse": (ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_int32, ct.c_void_p, ct.c_void_p]),
    "prop_apply_operator": (ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_void_p, ct.c_void_p]),
    "prop_get_correction": (ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_int32, ct.c_void_p]),
    "prop_set_guess_net": (ct.c_int, [ct.c_void_p, ct.c_int32, ct.POINTER(ct.c_int32), ct.c_void_p, ct.c_void_p]),
    "prop_get_net_io": (ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_int32, ct.c_void_p, ct.c_void_p]),
    "prop_fft2_noalloc": (ct.c_int, [ct.c_int32, ct.c_int32, ct.c_int32, ct.c_int32, ct.c_int32, ct.c_void_p,
                                     ct.c_void_p]),
    "prop_selftest_wait_timeout": (ct.c_int, [ct.c_void_p]),
    # learned initial guess (include/prop_cnn.h)
    "prop_cnn_conv": (ct.c_int, [ct.c_int32, ct.c_int32, ct.c_int32, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                 ct.c_void_p, ct.c_int32, ct.c_int32, ct.c_int32, ct.c_void_p, ct.c_int32,
                                 ct.c_int32, ct.c_void_p]),
    "prop_cnn_wgrad_workspace": (ct.c_int, [ct.c_int32, ct.c_int32, ct.c_int32, ct.c_int32, ct.c_int32,
                                            ct.POINTER(ct.c_size_t)]),
    "prop_cnn_wgrad": (ct.c_int, [ct.c_int32, ct.c_int32, ct.c_void_p, ct.c_void_p, ct.c_int32, ct.c_int32,
                                  ct.c_int32, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_size_t, ct.c_void_p]),
    "prop_cnn_flip_transpose": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int32, ct.c_int32, ct.c_void_p]),
    "prop_cnn_relu_mask": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int64, ct.c_void_p]),
    "prop_cnn_to_bf16": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int64, ct.c_void_p]),
    "prop_cnn_mse": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int64, ct.c_int32, ct.c_int32,
                                ct.c_void_p, ct.c_void_p]),
    "prop_cnn_set_path": (ct.c_int, [ct.c_int32]),
    "prop_cnn_check": (ct.c_int, [ct.c_void_p]),
    "prop_cnn_adam": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int64, ct.c_float,
                                 ct.c_float, ct.c_float, ct.c_float, ct.c_int32, ct.c_void_p, ct.c_void_p]),
}


def lib():
    """The loaded libprop.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2410_17446_gb300.build.build()")
        L = ct.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class PropError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().prop_error_string(status).decode()
        super().__init__(f"{where}: {msg} (status {status})")


def check(status: int, where: str) -> None:
    if status != PROP_OK:
        raise PropError(status, where)


def _dptr(buf) -> int:
    """Address of a torch tensor or numpy array (host)."""
    if hasattr(buf, "data_ptr"):
        return buf.data_ptr()
    return buf.ctypes.data


# ---- same-named thin wrappers ----------------------------------------------

def prop_default_opts(ncomp: int, precision: int) -> prop_opts:
    o = prop_opts()
    check(lib().prop_default_opts(ct.byref(o), ncomp, precision), "prop_default_opts")
    return o


def prop_workspace_size(grids: Sequence[prop_grid], npoles: int, opts: prop_opts) -> int:
    arr = (prop_grid * len(grids))(*grids)
    n = ct.c_size_t()
    check(lib().prop_workspace_size(len(grids), arr, npoles, ct.byref(opts), ct.byref(n)), "prop_workspace_size")
    return n.value


def prop_fft2_workspace_size(nx: int, ny: int, precision: int) -> int:
    n = ct.c_size_t()
    check(lib().prop_fft2_workspace_size(nx, ny, precision, ct.byref(n)), "prop_fft2_workspace_size")
    return n.value


def prop_fft2(nx, ny, batch, precision, inverse, d_data, d_work, work_bytes, stream=0) -> None:
    check(lib().prop_fft2(nx, ny, batch, precision, inverse, _dptr(d_data), _dptr(d_work), work_bytes,
                          stream), "prop_fft2")


def prop_get_fft_plan(n: int, precision: int) -> prop_fft_plan:
    p = prop_fft_plan()
    check(lib().prop_get_fft_plan(n, precision, ct.byref(p)), "prop_get_fft_plan")
    return p


def prop_set_fft_plan(n: int, precision: int, rows: int, cols: int, rows_small: Optional[int] = None,
                      cols_small: Optional[int] = None) -> None:
    """Large launches use (rows, cols); launches of at most PROP_FFT_SMALL_ITEMS arrays use
    (rows_small, cols_small), by default the same."""
    p = prop_fft_plan(rows, cols, rows if rows_small is None else rows_small, cols if cols_small is None else cols_small)
    check(lib().prop_set_fft_plan(n, precision, ct.byref(p)), "prop_set_fft_plan")


def prop_fft_autotune_workspace_size(n: int, precision: int, batch: int) -> int:
    b = ct.c_size_t()
    check(lib().prop_fft_autotune_workspace_size(n, precision, batch, ct.byref(b)), "prop_fft_autotune_workspace_size")
    return b.value


def prop_fft_autotune(n, precision, batch, reps, d_work, work_bytes, stream=0, l2cold=1):
    """Returns (best plan, round-trip times in ms indexed 3 rows + cols)."""
    best = prop_fft_plan()
    ms = (ct.c_float * 6)()
    check(lib().prop_fft_autotune(n, precision, batch, reps, l2cold, _dptr(d_work), work_bytes, stream, ct.byref(best),
                                  ms), "prop_fft_autotune")
    return best, list(ms)


def prop_fft2_noalloc(nx, ny, batch, precision, inverse, d_data, stream=0) -> None:
    """prop_fft2 without a caller workspace, for callers that cannot allocate device memory."""
    check(lib().prop_fft2_noalloc(nx, ny, batch, precision, inverse, _dptr(d_data), stream), "prop_fft2_noalloc")


class Propagator:
    """Owns one handle and its torch-allocated workspace."""

    def __init__(self, grids, k0: float, n0: float, dz: float, poles, residues, r0,
                 ncomp: int = 1, precision: int = PROP_FP32, restart: int = 20, max_restarts: Optional[int] = None,
                 tol: Optional[float] = None, device: str = "cuda", stream=None, guess: int = PROP_GUESS_ZERO,
                 precond: Optional[int] = None, form: int = PROP_FORM_EXPONENTIAL, substeps: int = 0,
                 multigroup: bool = True):
        import torch
        self.torch = torch
        self.grids = [prop_grid(int(g[0]), int(g[1]), float(g[2]), float(g[3])) if not isinstance(g, prop_grid)
                      else g for g in grids]
        self.nbeams = len(self.grids)
        self.ncomp = ncomp
        self.opts = prop_default_opts(ncomp, precision)
        self.opts.restart = restart
        if max_restarts is not None:
            self.opts.max_restarts = max_restarts
        if tol is not None:
            self.opts.tol = tol
        self.opts.guess = guess
        if precond is not None:
            self.opts.precond = precond
        self.opts.form = form
        self.opts.substeps = substeps
        self.opts.multigroup = 1 if multigroup else 0
        poles = np.asarray(poles, np.complex128)
        residues = np.asarray(residues, np.complex128)
        self.npoles = poles.size
        self.ws_bytes = prop_workspace_size(self.grids, self.npoles, self.opts)
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=device)
        s = stream if stream is not None else torch.cuda.current_stream(device)
        self.stream = s
        pr = np.ascontiguousarray(np.stack([poles.real, poles.imag], -1).ravel())
        rr = np.ascontiguousarray(np.stack([residues.real, residues.imag], -1).ravel())
        r0a = np.array([np.real(r0), np.imag(r0)], np.float64)
        arr = (prop_grid * self.nbeams)(*self.grids)
        h = ct.c_void_p()
        check(lib().prop_create(self.nbeams, arr, k0, n0, dz, self.npoles,
                                pr.ctypes.data_as(ct.POINTER(ct.c_double)),
                                rr.ctypes.data_as(ct.POINTER(ct.c_double)),
                                r0a.ctypes.data_as(ct.POINTER(ct.c_double)), ct.byref(self.opts),
                                self.workspace.data_ptr(), self.ws_bytes, s.cuda_stream, ct.byref(h)),
              "prop_create")
        self.h = h

    @classmethod
    def from_table(cls, grids, k0, n0, dz, table: dict, **kw):
        poles = np.array([complex(a, b) for a, b in table["poles"]])
        res = np.array([complex(a, b) for a, b in table["residues"]])
        return cls(grids, k0, n0, dz, poles, res, complex(*table["r0"]), **kw)

    def shape(self, beam: int):
        g = self.grids[beam]
        return (self.ncomp, g.ny, g.nx)

    def set_medium(self, beam: int, n2) -> None:
        check(lib().prop_set_medium(self.h, beam, _dptr(n2)), "prop_set_medium")

    def set_field(self, beam: int, w) -> None:
        check(lib().prop_set_field(self.h, beam, _dptr(w)), "prop_set_field")

    def get_field(self, beam: int, out=None):
        if out is None:
            out = np.empty(self.shape(beam), np.complex128)
        check(lib().prop_get_field(self.h, beam, _dptr(out)), "prop_get_field")
        return out

    def get_e3(self, beam: int, out=None):
        """E3 recovered from Gauss's law for the beam's current field (vector handles)."""
        if out is None:
            g = self.grids[beam]
            out = np.empty((g.ny, g.nx), np.complex128)
        check(lib().prop_get_e3(self.h, beam, _dptr(out)), "prop_get_e3")
        return out

    @property
    def substeps(self) -> int:
        """Runge-Kutta steps per dz of a pseudo-differential handle (0 for the exponential form)."""
        v = ct.c_int32()
        check(lib().prop_get_substeps(self.h, ct.byref(v)), "prop_get_substeps")
        return v.value

    def step(self) -> None:
        check(lib().prop_step(self.h), "prop_step")

    def run(self, nsteps: int, medium_cb=None) -> None:
        if medium_cb is None:
            cb = MEDIUM_FN(0)
        else:
            cb = MEDIUM_FN(lambda h, s, u: int(medium_cb(s) or 0))
        self._cb = cb
        check(lib().prop_run(self.h, nsteps, cb, None), "prop_run")

    def stats(self) -> prop_stats:
        st = prop_stats()
        check(lib().prop_get_stats(self.h, ct.byref(st)), "prop_get_stats")
        return st

    def iterations(self) -> np.ndarray:
        out = np.zeros(self.nbeams * self.npoles, np.int32)
        check(lib().prop_get_iterations(self.h, out.ctypes.data_as(ct.POINTER(ct.c_int32))), "prop_get_iterations")
        return out.reshape(self.nbeams, self.npoles)

    def set_profiling(self, on: bool) -> None:
        check(lib().prop_set_profiling(self.h, 1 if on else 0), "prop_set_profiling")

    def profile(self) -> dict:
        arr = (prop_kernel_profile * PROP_NKINDS)()
        check(lib().prop_get_profile(self.h, arr), "prop_get_profile")
        return {a.name.decode(): {"launches": a.launches, "total_ms": a.total_ms, "alg_bytes": a.alg_bytes}
                for a in arr}

    def apply_freespace_inverse(self, beam: int, pole: int, d_v, d_out) -> None:
        check(lib().prop_apply_freespace_inverse(self.h, beam, pole, _dptr(d_v), _dptr(d_out)),
              "prop_apply_freespace_inverse")

    def set_guess_net(self, channels, weights, biases) -> None:
        """weights: per layer float arrays [9, co, ci] (rounded to bf16 here); biases: per layer [co]."""
        import torch
        ch = (ct.c_int32 * len(channels))(*channels)
        wb = torch.cat([torch.as_tensor(np.asarray(w, np.float32)).reshape(-1) for w in weights]).to(torch.bfloat16)
        bb = torch.cat([torch.as_tensor(np.asarray(b, np.float32)).reshape(-1) for b in biases])
        wb, bb = wb.contiguous(), bb.contiguous()
        check(lib().prop_set_guess_net(self.h, len(channels) - 1, ch, wb.data_ptr(), bb.data_ptr()),
              "prop_set_guess_net")

    def get_net_io(self, beam: int, pole: int, d_in_bf16, d_target) -> None:
        check(lib().prop_get_net_io(self.h, beam, pole, _dptr(d_in_bf16), _dptr(d_target)), "prop_get_net_io")

    def get_correction(self, beam: int, pole: int, out=None):
        if out is None:
            out = np.empty(self.shape(beam), np.complex128)
        check(lib().prop_get_correction(self.h, beam, pole, _dptr(out)), "prop_get_correction")
        return out

    def apply_operator(self, beam: int, d_v, d_out) -> None:
        check(lib().prop_apply_operator(self.h, beam, _dptr(d_v), _dptr(d_out)), "prop_apply_operator")

    def close(self) -> None:
        if getattr(self, "h", None):
            lib().prop_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
