"""Pins of the oracle's Newton iterations.

* all-at-once Newton (eq. 4-7) converges to the sequential BDF1 solution
  (Sec. 2) to 1e-12 -- two different algorithms for the same discrete system;
* the first level's all-at-once iterates equal the sequential first step's
  Newton iterates (block lower-triangular structure of eq. 6);
* quadratic convergence (Sec. 8.1: the iterations converge quadratically);
* first-order temporal convergence on a field the spatial stencils represent
  exactly (so the only error is BDF1's).
"""
import numpy as np
import pytest

import oracle
from paper_2406_00878_gb300 import workloads as W
from tests.fields import boundary_levels, on_nodes


@pytest.mark.parametrize("make", [
    lambda: W.heat32(0),
    lambda: W.random_problem(4, 9, 7, 6, W.BURGERS, with_bc=True, with_q=True),
    lambda: W.random_problem(5, 8, 10, 5, W.HEAT, with_bc=True, with_q=True),
    lambda: W.truncated(W.burgers256(0), 2),
])
def test_all_at_once_equals_sequential_bdf1(make):
    p = make()
    U, it, res, _ = oracle.solve(p, tol=1e-13)
    Useq, iters = oracle.sequential_bdf1(p.grid, p.params, p.M, p.dt, p.u0, p.bc, p.q, tol=1e-14)
    scale = np.abs(Useq).max()
    assert np.abs(U - Useq).max() <= 1e-12 * scale
    assert it >= 2 and np.all(iters >= 1)


def test_first_level_iterates_equal_sequential_first_step():
    p = W.random_problem(6, 6, 5, 4, W.HEAT, with_bc=True)
    g, Ns = p.grid, p.grid.ns
    u = p.u0.copy()
    bnd = p.bc[0]
    for k in range(1, 4):
        # k sequential Newton updates on level 1 from the guess u^0
        r = oracle.level_residual(g, p.params, p.dt, p.u0, u, bnd)
        cf = oracle.level_jacobian(g, p.params, p.dt, u, bnd)
        u = u + oracle.level_solve(g.nx, g.ny, cf, r)
        Uk, it, _, _ = oracle.newton_all_at_once(g, p.params, p.M, p.dt, p.u0, p.plain_guess(), p.bc, p.q,
                                                 tol=0.0, maxit=k)
        np.testing.assert_allclose(Uk[0], u, rtol=0, atol=1e-13)


def test_newton_converges_quadratically_on_heat32():
    p = W.heat32(0)
    U, it, res, upd = oracle.solve(p, tol=1e-13)
    # order estimates p_k = log(r_{k+1}/r_k) / log(r_k/r_{k-1}) while the residual
    # is above round-off; the last one must be ~2
    live = [r for r in res if r > 1e-12]
    orders = [np.log(live[k + 1] / live[k]) / np.log(live[k] / live[k - 1]) for k in range(1, len(live) - 1)]
    assert 1.8 < orders[-1] < 2.3, (res, orders)
    assert res[-1] <= 1e-13


def _scalar_bdf1(a0, c, dt):
    """BDF1 for a' + 2 a^2 = c(t): (a_n - a_{n-1})/dt + 2 a_n^2 = c_n, positive root."""
    out, prev = [], a0
    for cn in c:
        prev = (-1.0 + np.sqrt(1.0 + 8.0 * dt * (prev + dt * cn))) / (4.0 * dt)
        out.append(prev)
    return np.array(out)


def test_spatially_exact_field_follows_scalar_bdf1_recursion():
    # u = a(t)(1 + x + y): for Burgers, f = u^2/2 is quadratic along x and y and the
    # Laplacian of u vanishes, so eq. 3's stencils are exact. With boundary data
    # a_n (1 + x + y) the discrete solution is exactly a_n (1 + x + y), where a_n is
    # BDF1 applied to the scalar ODE a' + 2 a^2 = c(t) -- solved in closed form.
    params = W.Params(W.BURGERS, 0.07, 0.0)
    M, dt = 12, 0.05
    g = W.Grid(6, 5, 0.0, 1.0, 0.0, 1.0)
    X, Y = g.nodes()
    s = (1.0 + X + Y).ravel()
    c = np.array([np.cos(n * dt) + 0.5 for n in range(1, M + 1)])
    an = _scalar_bdf1(0.8, c, dt)
    bc = np.array([a * np.concatenate(_boundary_s(g)) for a in an])
    p = W.Problem("lin", g, params, M, dt, 0.8 * s, bc, c[:, None] * s[None, :])
    U, it, res, _ = oracle.solve(p, tol=1e-14)
    np.testing.assert_allclose(U, an[:, None] * s[None, :], rtol=0, atol=1e-13)


def _boundary_s(g):
    xs = g.xl + g.hx * np.arange(1, g.nx + 1)
    ys = g.yl + g.hy * np.arange(1, g.ny + 1)
    return [1.0 + xs + g.yl, 1.0 + xs + g.yr, 1.0 + g.xl + ys, 1.0 + g.xr + ys]


def test_first_order_in_time_on_spatially_exact_field():
    # Same field with exact data a(t) = exp(-t): the error against the exact solution
    # is BDF1's time error and must fall as dt^1.
    params = W.Params(W.BURGERS, 0.07, 0.0)
    a = lambda t: np.exp(-t)
    ap = lambda t: -np.exp(-t)
    fn = lambda x, y, t: a(t) * (1.0 + x + y)
    errs, dts = [], []
    for M in (8, 16, 32, 64):
        g = W.Grid(6, 5, 0.0, 1.0, 0.0, 1.0)
        dt = 1.0 / M
        X, Y = g.nodes()
        s = (1.0 + X + Y).ravel()
        q = np.array([(ap(n * dt) + 2 * a(n * dt) ** 2) * s for n in range(1, M + 1)])
        p = W.Problem("lin", g, params, M, dt, on_nodes(g, fn, 0.0), boundary_levels(g, fn, M, dt), q)
        U, it, res, _ = oracle.solve(p, tol=1e-14)
        exact = np.array([on_nodes(g, fn, n * dt) for n in range(1, M + 1)])
        errs.append(np.abs(U - exact).max())
        dts.append(dt)
    orders = [np.log(errs[k - 1] / errs[k]) / np.log(dts[k - 1] / dts[k]) for k in range(1, len(errs))]
    assert all(0.9 < o < 1.1 for o in orders), (errs, orders)
