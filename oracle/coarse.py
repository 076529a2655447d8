"""FP64 CPU oracle for the paper's initial guess (Sec. 4, end of the section on the
decoupled systems): solve the problem sequentially on a grid coarsened by c_f in
each spatial direction and in time, then interpolate the coarse solution back to the
fine space-time grid with 1-D cubic splines.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` alone. Shares no code with the
CUDA library.

Readings where the paper is silent (the same readings the library takes):

* coarse grid: ``nx_c = (nx + 1) // c_f - 1`` interior nodes in x (the same in y) on
  the same domain, and ``M_c = M // c_f`` levels of step ``M dt / M_c`` (same end time);
* coarse data: u^0 and the sources bilinear in space between the fine interior nodes,
  the Dirichlet data linear along each edge; sources and Dirichlet data linear in time
  between fine levels (all of these are injections where coarse and fine nodes meet);
* the coarse problem is solved by sequential BDF1 (oracle O1);
* splines are natural cubic splines (zero second derivative at both ends), taken along
  x (knots: the west edge value, the coarse nodes, the east edge value), then y (knots:
  south edge value, the x-interpolated rows, north edge value), then t (knots: u^0 at
  t = 0 and the coarse levels). The paper names splines per spatial coordinate only; the
  time direction, which it also coarsens, takes the same kind of spline.

Parity status: pinned by ``tests/test_oracle_coarse.py`` (exact reproduction of
discrete solutions that are linear in space and time, injection at coincident nodes,
fourth-order spline convergence for data with zero end curvature).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np
from scipy.interpolate import CubicSpline

from . import sequential_bdf1


@dataclass(frozen=True)
class _Grid:
    nx: int
    ny: int
    xl: float
    xr: float
    yl: float
    yr: float


def coarse_sizes(nx: int, ny: int, M: int, cf: int):
    """(nx_c, ny_c, M_c) of the grid coarsened by cf; raises ValueError when a size drops below 1."""
    if cf < 2:
        raise ValueError("coarsening factor must be at least 2")
    nxc, nyc, Mc = (nx + 1) // cf - 1, (ny + 1) // cf - 1, M // cf
    if nxc < 1 or nyc < 1 or Mc < 1:
        raise ValueError(f"grid {nx}x{ny}x{M} too small to coarsen by {cf}")
    return nxc, nyc, Mc


def _interior_x(n, lo, hi):
    """Coordinates of the n interior nodes of [lo, hi]."""
    return lo + (hi - lo) / (n + 1) * np.arange(1, n + 1)


def _bilinear(f, grid, gc):
    """Values of f (ny, nx) on the fine interior nodes, linearly interpolated in x and then
    in y at the coarse interior nodes."""
    xf, yf = _interior_x(grid.nx, grid.xl, grid.xr), _interior_x(grid.ny, grid.yl, grid.yr)
    xc, yc = _interior_x(gc.nx, gc.xl, gc.xr), _interior_x(gc.ny, gc.yl, gc.yr)
    rows = np.array([np.interp(xc, xf, f[j]) for j in range(grid.ny)])            # (ny, nxc)
    return np.array([np.interp(yc, yf, rows[:, i]) for i in range(gc.nx)]).T      # (nyc, nxc)


def _edges(b, grid, gc):
    """One level of Dirichlet data (south nx, north nx, west ny, east ny), linear along
    each edge, at the coarse edge nodes."""
    nx, ny = grid.nx, grid.ny
    xf, yf = _interior_x(nx, grid.xl, grid.xr), _interior_x(ny, grid.yl, grid.yr)
    xc, yc = _interior_x(gc.nx, gc.xl, gc.xr), _interior_x(gc.ny, gc.yl, gc.yr)
    S, N, Wst, E = b[:nx], b[nx:2 * nx], b[2 * nx:2 * nx + ny], b[2 * nx + ny:]
    return np.concatenate([np.interp(xc, xf, S), np.interp(xc, xf, N), np.interp(yc, yf, Wst), np.interp(yc, yf, E)])


def _at_time(levels, t, dt):
    """Linear interpolation in time of per-level data levels[n] (time (n + 1) dt) at time t >= dt."""
    M = levels.shape[0]
    s = t / dt                       # 1-based fine level position
    n0 = min(max(int(np.floor(s)), 1), M)
    n1 = min(n0 + 1, M)
    w = min(max(s - n0, 0.0), 1.0)
    return (1.0 - w) * levels[n0 - 1] + w * levels[n1 - 1]


def restrict(grid, M, dt, u0, bc, q, cf):
    """The coarse problem: (coarse grid, M_c, dt_c, u0_c, bc_c or None, q_c or None)."""
    nxc, nyc, Mc = coarse_sizes(grid.nx, grid.ny, M, cf)
    gc = _Grid(nxc, nyc, grid.xl, grid.xr, grid.yl, grid.yr)
    T = M * dt
    dtc = T / Mc
    u0c = _bilinear(np.asarray(u0, dtype=np.float64).reshape(grid.ny, grid.nx), grid, gc).ravel()
    bcc = qc = None
    if bc is not None:
        bc = np.asarray(bc, dtype=np.float64).reshape(M, -1)
        bcc = np.array([_edges(_at_time(bc, l * dtc, dt), grid, gc) for l in range(1, Mc + 1)])
    if q is not None:
        q = np.asarray(q, dtype=np.float64).reshape(M, grid.ny, grid.nx)
        qc = np.array([_bilinear(_at_time(q, l * dtc, dt), grid, gc).ravel() for l in range(1, Mc + 1)])
    return gc, Mc, dtc, u0c, bcc, qc


def interpolate(grid, M, dt, u0, bc, gc, Mc, Uc, bcc):
    """Natural cubic splines along x, y and t from the coarse solution Uc (Mc, nsc) to the
    fine space-time grid; returns U (M, Ns)."""
    nx, ny = grid.nx, grid.ny
    T = M * dt
    xf, yf = _interior_x(nx, grid.xl, grid.xr), _interior_x(ny, grid.yl, grid.yr)
    xk = np.concatenate([[gc.xl], _interior_x(gc.nx, gc.xl, gc.xr), [gc.xr]])
    yk = np.concatenate([[gc.yl], _interior_x(gc.ny, gc.yl, gc.yr), [gc.yr]])
    Uc = np.asarray(Uc, dtype=np.float64).reshape(Mc, gc.ny, gc.nx)
    bcf = None if bc is None else np.asarray(bc, dtype=np.float64).reshape(M, -1)
    levels = np.empty((Mc, ny, nx))
    for l in range(Mc):
        tl = (l + 1) * T / Mc
        # x: one spline per coarse row, through the west/east Dirichlet values of the coarse problem
        rows = np.empty((gc.ny, nx))
        for j in range(gc.ny):
            w = 0.0 if bcc is None else bcc[l][2 * gc.nx + j]
            e = 0.0 if bcc is None else bcc[l][2 * gc.nx + gc.ny + j]
            rows[j] = CubicSpline(xk, np.concatenate([[w], Uc[l, j], [e]]), bc_type="natural")(xf)
        # y: one spline per fine column, through the fine south/north Dirichlet values at t_l
        b = None if bcf is None else _at_time(bcf, tl, dt)
        for i in range(nx):
            s = 0.0 if b is None else b[i]
            n = 0.0 if b is None else b[nx + i]
            levels[l, :, i] = CubicSpline(yk, np.concatenate([[s], rows[:, i], [n]]), bc_type="natural")(yf)
    # t: one spline per fine node, knots t = 0 (u^0) and t_l = l T / M_c
    tk = np.arange(Mc + 1) * (T / Mc)
    tf = np.arange(1, M + 1) * dt
    data = np.concatenate([np.asarray(u0, dtype=np.float64).reshape(1, ny * nx), levels.reshape(Mc, ny * nx)])
    return CubicSpline(tk, data, axis=0, bc_type="natural")(tf)


def coarse_guess(grid, params, M, dt, u0, bc=None, q=None, cf=3, tol=1e-14):
    """The paper's initial iterate: restrict, solve the coarse problem sequentially (O1),
    interpolate. Returns (U (M, Ns), coarse solution (M_c, nsc), coarse grid)."""
    gc, Mc, dtc, u0c, bcc, qc = restrict(grid, M, dt, u0, bc, q, cf)
    Uc, _ = sequential_bdf1(gc, params, Mc, dtc, u0c, bcc, qc, tol=tol)
    return interpolate(grid, M, dt, u0, bc, gc, Mc, Uc, bcc), Uc, gc
