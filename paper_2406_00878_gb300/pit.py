"""ctypes binding of libpit.so (C ABI in include/pit.h), same names as the ABI.

Argument marshalling only: every step of the method runs in the CUDA library.
Device arrays are torch tensors (float64, contiguous, on the context's device);
host arrays for ``pit_solve_host`` are numpy float64 arrays (or CPU tensors).
A failing call raises ``PitError`` carrying the status and ``pit_last_error``.
The library is loaded on first use and the call fails loudly if it is missing.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

from . import build as _build

(PIT_OK, PIT_EINVAL, PIT_ECUDA, PIT_ENOMEM, PIT_ENOCONV, PIT_EDIVERGED, PIT_ETIMEOUT, PIT_EUNSUPPORTED,
 PIT_EBOUNDS) = range(9)
PIT_HEAT, PIT_BURGERS = 0, 1
PIT_LIN_AUTO, PIT_LIN_SOR, PIT_LIN_BICGSTAB = 0, 1, 2
PIT_FP64, PIT_FP32_INNER = 0, 1
PIT_START_PLAIN, PIT_START_GIVEN = 0, 1
PIT_MAX_NEWTON = 64
PIT_NOALLOC_MAX_NX, PIT_NOALLOC_MAX_TEAM, PIT_NOALLOC_MAX_LEVELS = 512, 160, 4096

#: every symbol include/pit.h declares
EXPORTS = ("pit_default_options", "pit_create", "pit_set_data", "pit_fill_plain_guess", "pit_coarse_guess",
           "pit_residual", "pit_assemble", "pit_block_solve", "pit_newton_step", "pit_solve", "pit_solve_host",
           "pit_last_error", "pit_status_string", "pit_destroy", "pit_block_solve_noalloc", "pit_batch_create",
           "pit_batch_solve", "pit_batch_result", "pit_batch_placement", "pit_batch_last_error", "pit_batch_destroy", "pit_net_param_count",
           "pit_net_create", "pit_net_get_params", "pit_net_set_params", "pit_net_guess", "pit_net_make_target",
           "pit_net_gradients", "pit_net_train_step", "pit_net_last_error", "pit_net_destroy",
           "pit_product_form_solve", "pit_solve_product", "pit_probe_fma_peak", "pit_conv3x3_forward",
           "pit_conv3x3_backward", "pit_wave_timers", "pit_bounds_status")


class pit_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("xl", ctypes.c_double), ("xr", ctypes.c_double),
                ("yl", ctypes.c_double), ("yr", ctypes.c_double)]


class pit_params(ctypes.Structure):
    _fields_ = [("equation", ctypes.c_int), ("mu_a", ctypes.c_double), ("mu_b", ctypes.c_double)]


class pit_options(ctypes.Structure):
    _fields_ = [("newton_max", ctypes.c_int), ("tol_res", ctypes.c_double), ("lin_solver", ctypes.c_int),
                ("eta_max", ctypes.c_double), ("eta_gamma", ctypes.c_double), ("lin_atol", ctypes.c_double),
                ("lin_max_iter", ctypes.c_int), ("sor_rho_max", ctypes.c_double), ("team_ctas", ctypes.c_int),
                ("wait_budget", ctypes.c_longlong), ("wave_teams", ctypes.c_int), ("precision", ctypes.c_int),
                ("window", ctypes.c_int), ("batch_wave_nodes", ctypes.c_int), ("window_start", ctypes.c_int)]


class pit_step_info(ctypes.Structure):
    _fields_ = [("res_inf", ctypes.c_double), ("upd_rms", ctypes.c_double), ("lin_iters_mean", ctypes.c_double),
                ("lin_iters_max", ctypes.c_int), ("levels_sor", ctypes.c_int), ("levels_capped", ctypes.c_int),
                ("ms_residual", ctypes.c_float), ("ms_assemble", ctypes.c_float), ("ms_solve", ctypes.c_float),
                ("us_halo_wait", ctypes.c_float), ("us_reduce_wait", ctypes.c_float), ("us_chain", ctypes.c_float)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class pit_solve_info(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int), ("converged", ctypes.c_int),
                ("res_inf", ctypes.c_double * (PIT_MAX_NEWTON + 1)), ("steps", pit_step_info * PIT_MAX_NEWTON),
                ("ms_total", ctypes.c_double), ("wave_teams", ctypes.c_int), ("wave_team_ctas", ctypes.c_int),
                ("wave_launches", ctypes.c_int), ("ms_wave", ctypes.c_float), ("us_pred_wait", ctypes.c_float),
                ("us_halo_wait", ctypes.c_float), ("us_reduce_wait", ctypes.c_float), ("windows", ctypes.c_int),
                ("newton_iters_total", ctypes.c_int), ("us_setup", ctypes.c_float), ("us_level_solve", ctypes.c_float),
                ("us_update", ctypes.c_float), ("windows_converged", ctypes.c_int),
                ("wave_ctas", ctypes.c_int)]

    def as_dict(self):
        k = self.newton_iters
        return {"newton_iters": k, "converged": bool(self.converged), "res_inf": list(self.res_inf[:k + 1]),
                "steps": [self.steps[i].as_dict() for i in range(k)], "ms_total": self.ms_total,
                "wave_teams": self.wave_teams, "wave_team_ctas": self.wave_team_ctas, "wave_ctas": self.wave_ctas,
                "wave_launches": self.wave_launches, "ms_wave": self.ms_wave, "us_pred_wait": self.us_pred_wait,
                "us_halo_wait": self.us_halo_wait, "us_reduce_wait": self.us_reduce_wait, "windows": self.windows,
                "newton_iters_total": self.newton_iters_total, "us_setup": self.us_setup,
                "us_level_solve": self.us_level_solve, "us_update": self.us_update,
                "windows_converged": self.windows_converged}


class pit_instance(ctypes.Structure):
    _fields_ = [("grid", pit_grid), ("M", ctypes.c_int), ("dt", ctypes.c_double), ("params", pit_params),
                ("u0_dev", ctypes.c_void_p), ("bc_dev", ctypes.c_void_p), ("q_dev", ctypes.c_void_p),
                ("U_dev", ctypes.c_void_p)]


class pit_batch_info(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int), ("ctas", ctypes.c_int), ("teams", ctypes.c_int), ("min_team", ctypes.c_int),
                ("max_team", ctypes.c_int), ("converged", ctypes.c_int), ("graph", ctypes.c_int),
                ("ms", ctypes.c_double), ("est_makespan_ms", ctypes.c_double), ("ms_tuning", ctypes.c_double),
                ("wave_jobs", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class pit_product_info(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("diagonals", ctypes.c_longlong), ("half_band", ctypes.c_longlong),
                ("min_pivot", ctypes.c_double), ("ms_assemble", ctypes.c_float), ("ms_products", ctypes.c_float),
                ("ms_factor", ctypes.c_float)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class pit_net_shape(ctypes.Structure):
    _fields_ = [("height", ctypes.c_int), ("width", ctypes.c_int), ("levels", ctypes.c_int),
                ("channels", ctypes.c_int), ("blocks", ctypes.c_int), ("max_batch", ctypes.c_int)]


class PitError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_status_name(status)}: {msg}")
        self.status = status


_lib = None
_lib_path: Optional[str] = None
_lock = threading.Lock()


def use_library(path: str) -> None:
    """Load the library from `path` instead of libpit.so (e.g. the bounds-checking build,
    ``build.build_check()``). Must come before the first call into the library."""
    global _lib_path
    with _lock:
        if _lib is not None and os.path.abspath(path) != os.path.abspath(_lib_path or _build.LIB):
            raise RuntimeError("use_library: the library is already loaded from another path")
        _lib_path = path


def lib():
    """Load libpit.so (building it first if needed); raises if it cannot be built or loaded."""
    global _lib, _lib_path
    with _lock:
        if _lib is None:
            path = _lib_path or _build.LIB
            if _lib_path is None and not os.path.exists(path):
                path = _build.build()
            _lib_path = path
            L = ctypes.CDLL(path)
            P, D, V = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p
            st = ctypes.c_int
            L.pit_default_options.argtypes = [ctypes.POINTER(pit_options)]
            L.pit_default_options.restype = None
            L.pit_create.argtypes = [ctypes.POINTER(pit_grid), ctypes.c_int, ctypes.c_double,
                                     ctypes.POINTER(pit_params), ctypes.POINTER(pit_options), V,
                                     ctypes.POINTER(P)]
            L.pit_create.restype = st
            L.pit_set_data.argtypes = [P, V, V, V]
            L.pit_set_data.restype = st
            L.pit_fill_plain_guess.argtypes = [P, V]
            L.pit_fill_plain_guess.restype = st
            L.pit_coarse_guess.argtypes = [P, ctypes.c_int, V, ctypes.POINTER(pit_solve_info)]
            L.pit_coarse_guess.restype = st
            L.pit_residual.argtypes = [P, V, V, D]
            L.pit_residual.restype = st
            L.pit_assemble.argtypes = [P, V, V]
            L.pit_assemble.restype = st
            L.pit_block_solve.argtypes = [P, V, V, V, ctypes.c_double, ctypes.POINTER(pit_step_info)]
            L.pit_block_solve.restype = st
            L.pit_newton_step.argtypes = [P, V, ctypes.POINTER(pit_step_info)]
            L.pit_newton_step.restype = st
            L.pit_solve.argtypes = [P, V, ctypes.POINTER(pit_solve_info)]
            L.pit_solve.restype = st
            L.pit_solve_host.argtypes = [P, V, V, ctypes.POINTER(pit_solve_info)]
            L.pit_solve_host.restype = st
            L.pit_last_error.argtypes = [P]
            L.pit_last_error.restype = ctypes.c_char_p
            L.pit_status_string.argtypes = [ctypes.c_int]
            L.pit_status_string.restype = ctypes.c_char_p
            L.pit_destroy.argtypes = [P]
            L.pit_destroy.restype = None
            L.pit_block_solve_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, V, V, V, ctypes.c_double,
                                                  ctypes.POINTER(pit_options), V, ctypes.c_char_p, ctypes.c_int]
            L.pit_block_solve_noalloc.restype = st
            L.pit_wave_timers.argtypes = [P, ctypes.POINTER(ctypes.c_ulonglong), ctypes.c_int]
            L.pit_wave_timers.restype = ctypes.c_int
            L.pit_probe_fma_peak.argtypes = [ctypes.c_int, V, D]
            L.pit_probe_fma_peak.restype = st
            L.pit_bounds_status.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
            L.pit_bounds_status.restype = st
            L.pit_batch_create.argtypes = [ctypes.POINTER(pit_instance), ctypes.c_int, ctypes.POINTER(pit_options), V,
                                           ctypes.POINTER(P)]
            L.pit_batch_create.restype = st
            L.pit_batch_solve.argtypes = [P, ctypes.POINTER(pit_batch_info)]
            L.pit_batch_solve.restype = st
            L.pit_batch_result.argtypes = [P, ctypes.c_int, D, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
            L.pit_batch_result.restype = st
            L.pit_batch_placement.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_int)]
            L.pit_batch_placement.restype = st
            L.pit_batch_last_error.argtypes = [P]
            L.pit_batch_last_error.restype = ctypes.c_char_p
            L.pit_batch_destroy.argtypes = [P]
            L.pit_batch_destroy.restype = None
            F = ctypes.POINTER(ctypes.c_float)
            NS = ctypes.POINTER(pit_net_shape)
            L.pit_net_param_count.argtypes = [NS]
            L.pit_net_param_count.restype = ctypes.c_longlong
            L.pit_net_create.argtypes = [NS, ctypes.c_ulonglong, V, ctypes.POINTER(P)]
            L.pit_net_create.restype = st
            L.pit_net_get_params.argtypes = [P, F]
            L.pit_net_get_params.restype = st
            L.pit_net_set_params.argtypes = [P, F]
            L.pit_net_set_params.restype = st
            L.pit_net_guess.argtypes = [P, V, F, ctypes.c_int, V]
            L.pit_net_guess.restype = st
            L.pit_net_make_target.argtypes = [P, V, V, V]
            L.pit_net_make_target.restype = st
            L.pit_net_gradients.argtypes = [P, V, F, V, ctypes.c_int, F, F]
            L.pit_net_gradients.restype = st
            L.pit_net_train_step.argtypes = [P, V, F, V, ctypes.c_int, ctypes.c_float, F]
            L.pit_net_train_step.restype = st
            L.pit_net_last_error.argtypes = [P]
            L.pit_net_last_error.restype = ctypes.c_char_p
            L.pit_net_destroy.argtypes = [P]
            L.pit_net_destroy.restype = None
            I = ctypes.c_int
            L.pit_conv3x3_forward.argtypes = [V, V, V, V, V, I, I, I, I, I, I, V]
            L.pit_conv3x3_forward.restype = st
            L.pit_conv3x3_backward.argtypes = [V, V, V, V, V, V, I, I, I, I, I, V]
            L.pit_conv3x3_backward.restype = st
            L.pit_product_form_solve.argtypes = [P, V, V, V, ctypes.POINTER(pit_product_info)]
            L.pit_product_form_solve.restype = st
            L.pit_solve_product.argtypes = [P, V, ctypes.POINTER(pit_solve_info)]
            L.pit_solve_product.restype = st
            _lib = L
        return _lib


def _status_name(s: int) -> str:
    try:
        return lib().pit_status_string(int(s)).decode()
    except Exception:
        return f"status {s}"


def _dptr(t, name: str, numel: Optional[int] = None):
    """Device pointer of a contiguous float64 CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a, name: str, numel: int):
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"] or a.size != numel:
            raise TypeError(f"{name} must be a contiguous float64 array of {numel} values")
        return ctypes.c_void_p(a.ctypes.data)
    import torch
    if isinstance(a, torch.Tensor) and not a.is_cuda and a.dtype == torch.float64 and a.is_contiguous() \
            and a.numel() == numel:
        return ctypes.c_void_p(a.data_ptr())
    raise TypeError(f"{name} must be a contiguous float64 host array of {numel} values")


class Context:
    """A pit_ctx handle plus its sizes; release with ``pit_destroy`` (or ``close``)."""

    def __init__(self, handle, grid: pit_grid, M: int):
        self.handle = handle
        self.nx, self.ny, self.M = grid.nx, grid.ny, M
        self.ns = grid.nx * grid.ny
        self.dof = self.ns * M

    def _check(self, status: int):
        if status != PIT_OK:
            raise PitError(status, lib().pit_last_error(self.handle).decode())

    def close(self):
        if self.handle:
            lib().pit_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pit_default_options() -> pit_options:
    o = pit_options()
    lib().pit_default_options(ctypes.byref(o))
    return o


def pit_create(grid, M: int, dt: float, params, opt: Optional[pit_options] = None, stream=None) -> Context:
    """grid/params: pit_grid/pit_params or any object with the same fields (e.g. workloads.Grid/Params).
    stream: a torch.cuda.Stream, an int handle, or None (torch's current stream)."""
    g = grid if isinstance(grid, pit_grid) else pit_grid(int(grid.nx), int(grid.ny), float(grid.xl),
                                                          float(grid.xr), float(grid.yl), float(grid.yr))
    p = params if isinstance(params, pit_params) else pit_params(int(params.equation), float(params.mu_a),
                                                                 float(params.mu_b))
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    elif not isinstance(stream, int):
        stream = stream.cuda_stream
    h = ctypes.c_void_p()
    s = lib().pit_create(ctypes.byref(g), int(M), float(dt), ctypes.byref(p),
                         ctypes.byref(opt) if opt is not None else None, ctypes.c_void_p(stream), ctypes.byref(h))
    if s != PIT_OK:
        raise PitError(s, "pit_create failed (see stderr)")
    return Context(h, g, int(M))


def pit_set_data(ctx: Context, u0, bc=None, q=None):
    ctx._check(lib().pit_set_data(ctx.handle, _dptr(u0, "u0", ctx.ns),
                                  _dptr(bc, "bc", ctx.M * (2 * ctx.nx + 2 * ctx.ny)), _dptr(q, "q", ctx.dof)))


def pit_fill_plain_guess(ctx: Context, U):
    ctx._check(lib().pit_fill_plain_guess(ctx.handle, _dptr(U, "U", ctx.dof)))


def pit_coarse_guess(ctx: Context, cf: int, U, check: bool = True):
    """The paper's coarse-grid + cubic-spline initial iterate into U. Returns (status,
    report of the coarse solve)."""
    info = pit_solve_info()
    s = lib().pit_coarse_guess(ctx.handle, int(cf), _dptr(U, "U", ctx.dof), ctypes.byref(info))
    if check:
        ctx._check(s)
    return s, info.as_dict()


def pit_residual(ctx: Context, U, R, want_norm: bool = True) -> Optional[float]:
    out = ctypes.c_double(0.0)
    ctx._check(lib().pit_residual(ctx.handle, _dptr(U, "U", ctx.dof), _dptr(R, "R", ctx.dof),
                                  ctypes.byref(out) if want_norm else None))
    return out.value if want_norm else None


def pit_assemble(ctx: Context, U, coef):
    ctx._check(lib().pit_assemble(ctx.handle, _dptr(U, "U", ctx.dof), _dptr(coef, "coef", 5 * ctx.dof)))


def pit_block_solve(ctx: Context, U, R, dU, eta: float = 1e-14) -> dict:
    info = pit_step_info()
    ctx._check(lib().pit_block_solve(ctx.handle, _dptr(U, "U", ctx.dof), _dptr(R, "R", ctx.dof),
                                     _dptr(dU, "dU", ctx.dof), float(eta), ctypes.byref(info)))
    return info.as_dict()


def pit_newton_step(ctx: Context, U) -> dict:
    info = pit_step_info()
    ctx._check(lib().pit_newton_step(ctx.handle, _dptr(U, "U", ctx.dof), ctypes.byref(info)))
    return info.as_dict()


def pit_solve(ctx: Context, U, check: bool = True):
    """Returns (status, info dict). Raises on failure when check is True."""
    info = pit_solve_info()
    s = lib().pit_solve(ctx.handle, _dptr(U, "U", ctx.dof), ctypes.byref(info))
    if check:
        ctx._check(s)
    return s, info.as_dict()


def pit_solve_host(ctx: Context, u0_host, U_host, check: bool = True):
    info = pit_solve_info()
    s = lib().pit_solve_host(ctx.handle, _hptr(u0_host, "u0_host", ctx.ns), _hptr(U_host, "U_host", ctx.dof),
                             ctypes.byref(info))
    if check:
        ctx._check(s)
    return s, info.as_dict()


def pit_product_form_solve(ctx: Context, U, R, dU, check: bool = True):
    """The literal eq. 8 product form (P^n du^n = r~^n, diagonally scaled, banded LU).
    Returns (status, info dict)."""
    info = pit_product_info()
    s = lib().pit_product_form_solve(ctx.handle, _dptr(U, "U", ctx.dof), _dptr(R, "R", ctx.dof),
                                     _dptr(dU, "dU", ctx.dof), ctypes.byref(info))
    if check:
        ctx._check(s)
    return s, info.as_dict()


def pit_solve_product(ctx: Context, U, check: bool = True):
    """Newton with the product-form block solve. Returns (status, info dict)."""
    info = pit_solve_info()
    s = lib().pit_solve_product(ctx.handle, _dptr(U, "U", ctx.dof), ctypes.byref(info))
    if check:
        ctx._check(s)
    return s, info.as_dict()


def pit_destroy(ctx: Context):
    ctx.close()


def pit_block_solve_noalloc(nx: int, ny: int, M: int, coef, R, dU, eta: float = 1e-14,
                            opt: Optional[pit_options] = None, stream=None, check: bool = True):
    """Context-free block solve from raw Jacobian entries that allocates nothing on the
    device (for callers that cannot allocate). Returns (status, message)."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    elif not isinstance(stream, int):
        stream = stream.cuda_stream
    dof = nx * ny * M
    buf = ctypes.create_string_buffer(512)
    s = lib().pit_block_solve_noalloc(int(nx), int(ny), int(M), _dptr(coef, "coef", 5 * dof), _dptr(R, "R", dof),
                                      _dptr(dU, "dU", dof), float(eta),
                                      ctypes.byref(opt) if opt is not None else None, ctypes.c_void_p(stream), buf,
                                      len(buf))
    msg = buf.value.decode()
    if check and s != PIT_OK:
        raise PitError(s, msg)
    return s, msg


WAVE_TIMER_NAMES = ("halo_wait_ns", "reduce_wait_ns", "pred_wait_ns", "total_ns", "setup_ns", "solve_ns",
                    "update_ns", "setup_load_ns", "setup_reduce_ns", "cells", "sweeps", "unused",
                    "sor_publish_cyc", "sor_interior_cyc", "sor_fetch_cyc", "sor_boundary_cyc", "sor_barrier5_cyc",
                    "sor_colour1_cyc", "sor_decide_cyc", "sor_barrier7_cyc", "setup_nodes_cyc", "setup_blockmax_cyc",
                    "setup_publish_cyc", "setup_teamreduce_cyc", "setup_fetch_cyc")


def pit_wave_timers(ctx: "Context") -> list:
    """Per-team phase timers of the last wavefront launch (list of dicts, one per team)."""
    n = len(WAVE_TIMER_NAMES) * 64  # up to 64 teams
    buf = (ctypes.c_ulonglong * n)()
    have = lib().pit_wave_timers(ctx.handle, buf, n)
    k = len(WAVE_TIMER_NAMES)
    return [dict(zip(WAVE_TIMER_NAMES, buf[t * k:(t + 1) * k])) for t in range(max(have, 0) // k)]


def pit_probe_fma_peak(precision: int = 0, stream=None) -> float:
    """Measured FMA rate of this GPU in TFLOP/s (precision 0 = FP64, 1 = FP32)."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    elif not isinstance(stream, int):
        stream = stream.cuda_stream
    out = ctypes.c_double(0.0)
    s = lib().pit_probe_fma_peak(int(precision), ctypes.c_void_p(stream), ctypes.byref(out))
    if s != PIT_OK:
        raise PitError(s, "pit_probe_fma_peak failed")
    return float(out.value)


# ------------------------------------------------------------- convenience

def pit_bounds_status() -> tuple:
    """(enabled, first_id): whether this library is the bounds-checking build, and the id of
    the first array a kernel indexed out of range since the last call (0 = none; cleared).
    Synchronises the device. Raises PitError when the device cannot be read."""
    en, fid = ctypes.c_int(0), ctypes.c_int(0)
    s = lib().pit_bounds_status(ctypes.byref(en), ctypes.byref(fid))
    if s not in (PIT_OK, PIT_EBOUNDS):
        raise PitError(s, "pit_bounds_status failed")
    return en.value, fid.value


def context_for(problem, opt: Optional[pit_options] = None, stream=None) -> Context:
    """Create a context for a workloads.Problem and upload its data (device tensors)."""
    import torch
    ctx = pit_create(problem.grid, problem.M, problem.dt, problem.params, opt, stream)
    dev = torch.device("cuda", torch.cuda.current_device())
    u0 = torch.as_tensor(np.ascontiguousarray(problem.u0), dtype=torch.float64, device=dev)
    bc = None if problem.bc is None else torch.as_tensor(np.ascontiguousarray(problem.bc), device=dev)
    q = None if problem.q is None else torch.as_tensor(np.ascontiguousarray(problem.q), device=dev)
    pit_set_data(ctx, u0, bc, q)
    torch.cuda.current_stream().synchronize()
    return ctx


class Batch:
    """A pit_batch handle plus the device tensors its problems point at (kept alive here)."""

    def __init__(self, handle, problems, tensors):
        self.handle = handle
        self.problems = problems
        self.tensors = tensors       # per problem: dict(u0=, bc=, q=, U=)

    def _check(self, status: int):
        if status != PIT_OK:
            raise PitError(status, lib().pit_batch_last_error(self.handle).decode())

    def close(self):
        if self.handle:
            lib().pit_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pit_batch_create(problems, opt: Optional[pit_options] = None, stream=None, U=None) -> Batch:
    """Upload a list of workloads.Problem and create a batch (runs the autotuner).
    U (optional): per problem a contiguous float64 CUDA tensor of M * Ns values that the
    batch solves into (and starts from, with window_start = PIT_START_GIVEN); by default
    the batch allocates them."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    elif not isinstance(stream, int):
        stream = stream.cuda_stream
    arr = (pit_instance * len(problems))()
    tensors = []
    for i, p in enumerate(problems):
        Ui = U[i] if U is not None else torch.empty(p.dof, dtype=torch.float64, device="cuda")
        _dptr(Ui, f"U[{i}]", p.dof)
        t = {"u0": torch.as_tensor(np.ascontiguousarray(p.u0), dtype=torch.float64, device="cuda"),
             "bc": None if p.bc is None else torch.as_tensor(np.ascontiguousarray(p.bc), device="cuda"),
             "q": None if p.q is None else torch.as_tensor(np.ascontiguousarray(p.q), device="cuda"),
             "U": Ui}
        tensors.append(t)
        g = p.grid
        arr[i].grid = pit_grid(int(g.nx), int(g.ny), float(g.xl), float(g.xr), float(g.yl), float(g.yr))
        arr[i].M = int(p.M)
        arr[i].dt = float(p.dt)
        arr[i].params = pit_params(int(p.params.equation), float(p.params.mu_a), float(p.params.mu_b))
        arr[i].u0_dev = t["u0"].data_ptr()
        arr[i].bc_dev = t["bc"].data_ptr() if t["bc"] is not None else None
        arr[i].q_dev = t["q"].data_ptr() if t["q"] is not None else None
        arr[i].U_dev = t["U"].data_ptr()
    torch.cuda.synchronize()
    h = ctypes.c_void_p()
    s = lib().pit_batch_create(arr, len(problems), ctypes.byref(opt) if opt is not None else None,
                               ctypes.c_void_p(stream), ctypes.byref(h))
    if s != PIT_OK:
        raise PitError(s, "pit_batch_create failed (see stderr)")
    return Batch(h, problems, tensors)


def pit_batch_solve(batch: Batch, check: bool = True):
    info = pit_batch_info()
    s = lib().pit_batch_solve(batch.handle, ctypes.byref(info))
    if check:
        batch._check(s)
    return s, info.as_dict()


def pit_batch_result(batch: Batch, i: int) -> dict:
    r = ctypes.c_double()
    it, wc, tc = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    batch._check(lib().pit_batch_result(batch.handle, int(i), ctypes.byref(r), ctypes.byref(it), ctypes.byref(wc),
                                        ctypes.byref(tc)))
    return {"res_inf": r.value, "newton_iters": it.value, "windows_converged": wc.value, "team_ctas": tc.value}


def pit_batch_placement(batch: Batch, i: int) -> dict:
    """How problem i is solved: `teams` teams of `team_ctas` CTAs (teams > 1: a wavefront
    job with that many Newton iterations in flight)."""
    te, tc = ctypes.c_int(), ctypes.c_int()
    batch._check(lib().pit_batch_placement(batch.handle, int(i), ctypes.byref(te), ctypes.byref(tc)))
    return {"teams": te.value, "team_ctas": tc.value}


def pit_batch_destroy(batch: Batch):
    batch.close()


# ------------------------------------------------------- learned initial guess

class Net:
    """A pit_net handle (the learned initial-guess network)."""

    def __init__(self, handle, shape: pit_net_shape):
        self.handle = handle
        self.shape = shape
        self.nparam = int(lib().pit_net_param_count(ctypes.byref(shape)))

    def _check(self, status: int):
        if status != PIT_OK:
            raise PitError(status, lib().pit_net_last_error(self.handle).decode())

    def close(self):
        if self.handle:
            lib().pit_net_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _fptr(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def pit_net_create(height, width, levels, channels=64, blocks=4, max_batch=16, seed=0, stream=None) -> Net:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    elif not isinstance(stream, int):
        stream = stream.cuda_stream
    shape = pit_net_shape(int(height), int(width), int(levels), int(channels), int(blocks), int(max_batch))
    h = ctypes.c_void_p()
    s = lib().pit_net_create(ctypes.byref(shape), ctypes.c_ulonglong(seed), ctypes.c_void_p(stream), ctypes.byref(h))
    if s != PIT_OK:
        raise PitError(s, "pit_net_create failed (see stderr)")
    return Net(h, shape)


def pit_net_get_params(net: Net) -> np.ndarray:
    out = np.empty(net.nparam, dtype=np.float32)
    net._check(lib().pit_net_get_params(net.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return out


def pit_net_set_params(net: Net, params):
    arr, ptr = _fptr(params)
    assert arr.size == net.nparam
    net._check(lib().pit_net_set_params(net.handle, ptr))


def pit_net_guess(net: Net, u0, lognu, U):
    """u0: float64 CUDA tensor [B, Ns]; lognu: B floats; U: float64 CUDA tensor [B, M, Ns] (out)."""
    B = len(lognu)
    arr, ptr = _fptr(lognu)
    net._check(lib().pit_net_guess(net.handle, _dptr(u0, "u0"), ptr, B, _dptr(U, "U")))


def pit_net_make_target(net: Net, u0, U, target):
    """target: a CUDA tensor of int16 / bfloat16 with H*W*M elements."""
    net._check(lib().pit_net_make_target(net.handle, _dptr(u0, "u0"), _dptr(U, "U"),
                                         ctypes.c_void_p(target.data_ptr())))


def pit_net_gradients(net: Net, u0, lognu, target, want_grads=True):
    B = len(lognu)
    arr, ptr = _fptr(lognu)
    loss = ctypes.c_float()
    grads = np.empty(net.nparam, dtype=np.float32) if want_grads else None
    net._check(lib().pit_net_gradients(net.handle, _dptr(u0, "u0"), ptr, ctypes.c_void_p(target.data_ptr()), B,
                                       ctypes.byref(loss),
                                       grads.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if want_grads else None))
    return loss.value, grads


def pit_net_train_step(net: Net, u0, lognu, target, lr, want_loss=False):
    B = len(lognu)
    arr, ptr = _fptr(lognu)
    loss = ctypes.c_float()
    net._check(lib().pit_net_train_step(net.handle, _dptr(u0, "u0"), ptr, ctypes.c_void_p(target.data_ptr()), B,
                                        ctypes.c_float(lr), ctypes.byref(loss) if want_loss else None))
    return loss.value if want_loss else None


def pit_net_destroy(net: Net):
    net.close()


def _tptr(t, name: str, dtype, numel: int):
    """Device pointer of a contiguous CUDA tensor of the given dtype and size (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous {dtype} CUDA tensor")
    if t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return ctypes.c_void_p(t.data_ptr())


def _stream_of(stream):
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def pit_conv3x3_forward(X, Wt, bias, res, Y, B, H, Wd, Cin, Cout, relu, stream=None):
    """One tensor-core conv layer: Y = act(conv3x3(X, Wt) + bias (+ res)), NHWC BF16."""
    import torch
    bf = torch.bfloat16
    n = B * H * Wd
    s = lib().pit_conv3x3_forward(_tptr(X, "X", bf, n * Cin), _tptr(Wt, "W", bf, Cout * 9 * Cin),
                                  _tptr(bias, "bias", torch.float32, Cout), _tptr(res, "res", bf, n * Cout),
                                  _tptr(Y, "Y", bf, n * Cout), B, H, Wd, Cin, Cout, int(bool(relu)),
                                  ctypes.c_void_p(_stream_of(stream)))
    if s != PIT_OK:
        raise PitError(s, "pit_conv3x3_forward failed")


def pit_conv3x3_backward(X, Wt, dY, dX, dW, db, B, H, Wd, Cin, Cout, stream=None):
    """Gradients of sum(dY * conv3x3(X, Wt)): dX (BF16, may be None), dW and db (FP32)."""
    import torch
    bf = torch.bfloat16
    n = B * H * Wd
    s = lib().pit_conv3x3_backward(_tptr(X, "X", bf, n * Cin), _tptr(Wt, "W", bf, Cout * 9 * Cin),
                                   _tptr(dY, "dY", bf, n * Cout), _tptr(dX, "dX", bf, n * Cin),
                                   _tptr(dW, "dW", torch.float32, Cout * 9 * Cin),
                                   _tptr(db, "db", torch.float32, Cout), B, H, Wd, Cin, Cout,
                                   ctypes.c_void_p(_stream_of(stream)))
    if s != PIT_OK:
        raise PitError(s, "pit_conv3x3_backward failed")
