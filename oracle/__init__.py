"""FP64 CPU oracle for the all-at-once BDF1 Newton method (arXiv 2406.00878).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA library: the arithmetic lives in ``pit_oracle.c`` (plain loops, IEEE
FP64, compiled with ``-ffp-contract=off``) and in the small dense numpy routines
below, which restate the paper's block algebra literally:

* ``dense_global_jacobian`` -- the block-bidiagonal matrix of eq. 6;
* ``product_form_solve``     -- Theorem 1 / eq. 8: P^n du^n = r~^n with the
  recursion P^{n+1} = P^n A_{n+1}, r~^{n+1} = P^n r^{n+1} + r~^n of Sec. 5;
* ``nonzero_diagonals``      -- the diagonal count of Remark 2 (Sec. 5);
* ``max_levels_cond_bound``  -- the largest N_t allowed by eq. 15 (Sec. 7).

Every function that takes a grid or params accepts any object with the fields
of ``paper_2406_00878_gb300.workloads.Grid`` / ``Params``.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, finite differences, brute-force dense solves, textbook
special cases (DST-I diagonalisation) or convergence orders.  The paper's own
table digits (grconv_heat, grconv_Burgers) are compared in rate only, because
the paper leaves the grid counting and the Burgers domain open.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pit_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libpit_oracle.so")
_OMP_PATH = os.path.join(_OUT_DIR, "libpit_oracle_omp.so")
_lock = threading.Lock()
_libs = {}
_use_omp = False

HEAT, BURGERS = 0, 1
SOLVER_AUTO, SOLVER_BAND_LU, SOLVER_BICGSTAB = 0, 1, 2


class _OgGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("xl", ctypes.c_double), ("xr", ctypes.c_double),
                ("yl", ctypes.c_double), ("yr", ctypes.c_double)]


class _OgParams(ctypes.Structure):
    _fields_ = [("equation", ctypes.c_int), ("mu_a", ctypes.c_double), ("mu_b", ctypes.c_double)]


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile pit_oracle.c with gcc into oracle/_build/libpit_oracle.so (single-threaded,
    the tested build) or, with openmp, libpit_oracle_omp.so (the timing build: the same
    arithmetic with the element-independent loops spread over threads)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    path = _OMP_PATH if openmp else _LIB_PATH
    if not force and os.path.exists(path) and os.path.getmtime(path) >= os.path.getmtime(_SRC):
        return path
    tmp = path + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
    cmd += ["-fopenmp"] if openmp else []
    cmd += ["-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


def use_threads(n: int) -> int:
    """Run the oracle's element-independent loops on n host threads (n > 1 loads the
    OpenMP timing build; n <= 1 the single-threaded build). Results are bitwise the
    same in both builds. Returns the thread count in use."""
    global _use_omp
    with _lock:
        _use_omp = n > 1
    if n > 1:
        return int(_L().oracle_set_threads(int(n)))
    return 1


def _L():
    return _load(_use_omp)


def _load(openmp: bool):
    with _lock:
        _lib = _libs.get(openmp)
        if _lib is None:
            _lib = ctypes.CDLL(build(openmp=openmp))
            _libs[openmp] = _lib
            D = ctypes.POINTER(ctypes.c_double)
            I = ctypes.POINTER(ctypes.c_int)
            G = ctypes.POINTER(_OgGrid)
            P = ctypes.POINTER(_OgParams)
            c_int, c_dbl, c_sz = ctypes.c_int, ctypes.c_double, ctypes.c_size_t
            sig = {
                "oracle_F": (None, [G, P, D, D, D]),
                "oracle_level_residual": (None, [G, P, c_dbl, D, D, D, D, D]),
                "oracle_residual": (None, [G, P, c_int, c_dbl, D, D, D, D, D]),
                "oracle_level_jacobian": (None, [G, P, c_dbl, D, D, D, D, D, D, D]),
                "oracle_jacobian": (None, [G, P, c_int, c_dbl, D, D, D]),
                "oracle_apply_A": (None, [c_int, c_int, D, c_sz, D, D]),
                "oracle_band_lu_solve": (c_int, [c_int, c_int, D, c_sz, D, D]),
                "oracle_bicgstab": (c_int, [c_int, c_int, D, c_sz, D, D, c_dbl, c_int]),
                "oracle_level_solve": (c_int, [c_int, c_int, D, c_sz, D, D, c_int, c_dbl]),
                "oracle_block_solve": (c_int, [c_int, c_int, c_int, D, D, D, c_int, c_dbl]),
                "oracle_newton_all_at_once": (c_int, [G, P, c_int, c_dbl, D, D, D, D, c_dbl, c_int, c_int, c_dbl, D,
                                                      D]),
                "oracle_sequential_bdf1": (c_int, [G, P, c_int, c_dbl, D, D, D, D, c_dbl, c_int, c_int, c_dbl, I]),
                "oracle_set_threads": (c_int, [c_int]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(_lib, name)
                fn.restype = res
                fn.argtypes = args
        return _lib


# --------------------------------------------------------------------- helpers

def _g(grid) -> _OgGrid:
    return _OgGrid(int(grid.nx), int(grid.ny), float(grid.xl), float(grid.xr), float(grid.yl), float(grid.yr))


def _p(params) -> _OgParams:
    return _OgParams(int(params.equation), float(params.mu_a), float(params.mu_b))


def _d(a):
    """Pointer to a C-contiguous float64 numpy array (or NULL for None)."""
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "oracle arrays must be contiguous float64"
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _arr(x, n=None):
    if x is None:
        return None
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None:
        assert a.size == n, (a.size, n)
    return a


# ------------------------------------------------------------ eq. 3 - eq. 6

def F(grid, params, u, bnd=None):
    """Spatial operator F of eq. 3 on one level (Ns values, x fastest)."""
    Ns = grid.nx * grid.ny
    u = _arr(u, Ns)
    bnd = _arr(bnd, 2 * grid.nx + 2 * grid.ny)
    out = np.empty(Ns)
    _L().oracle_F(ctypes.byref(_g(grid)), ctypes.byref(_p(params)), _d(u), _d(bnd), _d(out))
    return out


def level_residual(grid, params, dt, u_prev, u, bnd=None, q=None):
    """r^n of eq. 5 for one level."""
    Ns = grid.nx * grid.ny
    out = np.empty(Ns)
    _L().oracle_level_residual(ctypes.byref(_g(grid)), ctypes.byref(_p(params)), float(dt), _d(_arr(u_prev, Ns)),
                               _d(_arr(u, Ns)), _d(_arr(bnd, 2 * grid.nx + 2 * grid.ny)), _d(_arr(q, Ns)), _d(out))
    return out


def residual(grid, params, M, dt, u0, U, bc=None, q=None):
    """All-at-once residual R = [r^1..r^M] (eq. 4-5); returns shape (M, Ns)."""
    Ns = grid.nx * grid.ny
    out = np.empty((M, Ns))
    _L().oracle_residual(ctypes.byref(_g(grid)), ctypes.byref(_p(params)), int(M), float(dt), _d(_arr(u0, Ns)),
                         _d(_arr(bc, M * (2 * grid.nx + 2 * grid.ny))), _d(_arr(q, M * Ns)), _d(_arr(U, M * Ns)),
                         _d(out))
    return out


def jacobian(grid, params, M, dt, U, bc=None):
    """Coefficients of A_1..A_M (eq. 5-6); returns shape (5, M, Ns) = C, W, E, S, N."""
    Ns = grid.nx * grid.ny
    out = np.empty((5, M, Ns))
    _L().oracle_jacobian(ctypes.byref(_g(grid)), ctypes.byref(_p(params)), int(M), float(dt),
                         _d(_arr(bc, M * (2 * grid.nx + 2 * grid.ny))), _d(_arr(U, M * Ns)), _d(out))
    return out


def level_jacobian(grid, params, dt, u, bnd=None):
    """Coefficients of one block A = I + dt dF/du at u; returns shape (5, Ns)."""
    Ns = grid.nx * grid.ny
    out = np.empty((5, Ns))
    _L().oracle_level_jacobian(ctypes.byref(_g(grid)), ctypes.byref(_p(params)), float(dt), _d(_arr(u, Ns)),
                               _d(_arr(bnd, 2 * grid.nx + 2 * grid.ny)), _d(out[0]), _d(out[1]), _d(out[2]),
                               _d(out[3]), _d(out[4]))
    return out


def apply_A(nx, ny, cf, x):
    """y = A x for one level; cf has shape (5, Ns)."""
    cf = _arr(cf, 5 * nx * ny)
    y = np.empty(nx * ny)
    _L().oracle_apply_A(nx, ny, _d(cf), nx * ny, _d(_arr(x, nx * ny)), _d(y))
    return y


def level_solve(nx, ny, cf, b, solver=SOLVER_AUTO, rtol=1e-14):
    """Solve one block A x = b (banded LU without pivoting, or BiCGStab)."""
    cf = _arr(cf, 5 * nx * ny)
    x = np.zeros(nx * ny)
    err = _L().oracle_level_solve(nx, ny, _d(cf), nx * ny, _d(_arr(b, nx * ny)), _d(x), int(solver), float(rtol))
    if err:
        raise RuntimeError("oracle level solve failed")
    return x


def bicgstab(nx, ny, cf, b, rtol=1e-14, maxit=100000, x0=None):
    """BiCGStab + Jacobi on one block; returns (x, iterations)."""
    cf = _arr(cf, 5 * nx * ny)
    x = np.zeros(nx * ny) if x0 is None else _arr(x0, nx * ny).copy()
    it = _L().oracle_bicgstab(nx, ny, _d(cf), nx * ny, _d(_arr(b, nx * ny)), _d(x), float(rtol), int(maxit))
    return x, it


def block_solve(nx, ny, M, coef, R, solver=SOLVER_AUTO, rtol=1e-14):
    """Exact block inverse of eq. 7 in nested form; coef (5, M, Ns), R (M, Ns) -> dU (M, Ns)."""
    Ns = nx * ny
    coef = _arr(coef, 5 * M * Ns)
    dU = np.empty((M, Ns))
    err = _L().oracle_block_solve(nx, ny, int(M), _d(coef), _d(_arr(R, M * Ns)), _d(dU), int(solver), float(rtol))
    if err:
        raise RuntimeError("oracle block solve failed")
    return dU


def newton_all_at_once(grid, params, M, dt, u0, U_init, bc=None, q=None, tol=1e-13, maxit=30,
                       solver=SOLVER_AUTO, lin_rtol=1e-14):
    """All-at-once Newton (eq. 4-7) from U_init. Returns (U, iterations, res_hist, upd_hist);
    iterations is -1 when tol was not reached."""
    Ns = grid.nx * grid.ny
    U = _arr(U_init, M * Ns).copy()
    res = np.full(maxit + 1, np.nan)
    upd = np.full(maxit + 1, np.nan)
    it = _L().oracle_newton_all_at_once(ctypes.byref(_g(grid)), ctypes.byref(_p(params)), int(M), float(dt),
                                        _d(_arr(u0, Ns)), _d(_arr(bc, M * (2 * grid.nx + 2 * grid.ny))),
                                        _d(_arr(q, M * Ns)), _d(U), float(tol), int(maxit), int(solver),
                                        float(lin_rtol), _d(res), _d(upd))
    n_res = (it + 1) if it >= 0 else int(np.sum(~np.isnan(res)))
    return U.reshape(M, Ns), it, res[:n_res], upd[:max(n_res - 1, 0)]


def sequential_bdf1(grid, params, M, dt, u0, bc=None, q=None, tol=1e-14, maxit=30, solver=SOLVER_AUTO,
                    lin_rtol=1e-14):
    """Sequential BDF1 time marching with Newton per step. Returns (U (M, Ns), iters per step)."""
    Ns = grid.nx * grid.ny
    U = np.empty(M * Ns)
    iters = np.zeros(M, dtype=np.int32)
    fail = _L().oracle_sequential_bdf1(ctypes.byref(_g(grid)), ctypes.byref(_p(params)), int(M), float(dt),
                                       _d(_arr(u0, Ns)), _d(_arr(bc, M * (2 * grid.nx + 2 * grid.ny))),
                                       _d(_arr(q, M * Ns)), _d(U), float(tol), int(maxit), int(solver),
                                       float(lin_rtol), iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if fail:
        raise RuntimeError(f"sequential BDF1 failed at step {fail}")
    return U.reshape(M, Ns), iters


def solve(problem, tol=1e-13, maxit=30, solver=SOLVER_AUTO, lin_rtol=1e-14, U_init=None):
    """Converged all-at-once solution of a workloads.Problem from the plain guess u^n = u^0."""
    Ns = problem.grid.nx * problem.grid.ny
    if U_init is None:
        U_init = np.tile(np.asarray(problem.u0, dtype=np.float64).reshape(1, Ns), (problem.M, 1))
    U, it, res, upd = newton_all_at_once(problem.grid, problem.params, problem.M, problem.dt, problem.u0, U_init,
                                         problem.bc, problem.q, tol=tol, maxit=maxit, solver=solver,
                                         lin_rtol=lin_rtol)
    if it < 0:
        raise RuntimeError(f"oracle Newton did not reach {tol}: history {res}")
    return U, it, res, upd


# --------------------------------------------- dense block algebra (tiny grids)

def dense_block(nx, ny, cf):
    """Dense Ns x Ns matrix of one 5-point block from its (5, Ns) coefficients."""
    Ns = nx * ny
    A = np.zeros((Ns, Ns))
    for j in range(ny):
        for i in range(nx):
            k = j * nx + i
            A[k, k] = cf[0][k]
            if i > 0:
                A[k, k - 1] = cf[1][k]
            if i < nx - 1:
                A[k, k + 1] = cf[2][k]
            if j > 0:
                A[k, k - nx] = cf[3][k]
            if j < ny - 1:
                A[k, k + nx] = cf[4][k]
    return A


def dense_global_jacobian(nx, ny, M, coef):
    """The block-bidiagonal space-time Jacobian of eq. 6: A_n on the diagonal, -I below."""
    Ns = nx * ny
    J = np.zeros((M * Ns, M * Ns))
    for n in range(M):
        J[n * Ns:(n + 1) * Ns, n * Ns:(n + 1) * Ns] = dense_block(nx, ny, coef[:, n, :])
        if n > 0:
            J[n * Ns:(n + 1) * Ns, (n - 1) * Ns:n * Ns] = -np.eye(Ns)
    return J


def product_form(nx, ny, M, coef, R):
    """Theorem 1 (eq. 8) by the recursion of Sec. 5: P^1 = A_1, r~^1 = r^1,
    P^{n+1} = P^n A_{n+1}, r~^{n+1} = P^n r^{n+1} + r~^n. Returns ([P^n], [r~^n])."""
    A = [dense_block(nx, ny, coef[:, n, :]) for n in range(M)]
    P = [A[0]]
    rt = [np.asarray(R[0], dtype=np.float64).copy()]
    for n in range(1, M):
        rt.append(P[n - 1] @ R[n] + rt[n - 1])
        P.append(P[n - 1] @ A[n])
    return P, rt


def product_form_solve(nx, ny, M, coef, R, diag_precondition=True):
    """Solve the decoupled systems P^n du^n = r~^n of eq. 8 level by level (dense LU),
    optionally with the diagonal preconditioner diag(P^n) of Sec. 7."""
    P, rt = product_form(nx, ny, M, coef, R)
    out = []
    for n in range(M):
        Pn, bn = P[n], rt[n]
        if diag_precondition:
            d = np.diag(Pn).copy()
            Pn = Pn / d[:, None]
            bn = bn / d
        out.append(np.linalg.solve(Pn, bn))
    return np.array(out)


def nonzero_diagonals(A, tol=0.0):
    """Number of distinct diagonals (column - row offsets) holding a nonzero of A (Remark 2)."""
    rows, cols = np.nonzero(np.abs(A) > tol)
    return len(np.unique(cols - rows))


def max_levels_cond_bound(N, mu, c=1.0, eps=1e-16):
    """Largest N_t that satisfies the condition-number bound of eq. 15 (Sec. 7):
    ((1 + 8 mu/(N_t h^2)) / (1 + 2 pi^2 mu/N_t))^N_t < c h^4 / eps with h = 1/N, tau = 1/N_t."""
    h = 1.0 / N
    rhs = c * h ** 4 / eps
    best = 0
    for nt in range(1, 100000):
        K = ((1.0 + 8.0 * mu / (nt * h * h)) / (1.0 + 2.0 * np.pi ** 2 * mu / nt)) ** nt
        if K < rhs:
            best = nt
        else:
            break
    return best
