"""Pins of the coarse-grid + cubic-spline initial guess oracle (the paper's initial
iterate, Sec. 4): discrete solutions that are linear in space and time survive every
step exactly, coarse data are injections where the grids meet, and the spline stage
converges at fourth order on data with zero end curvature."""
import numpy as np
import pytest

import oracle
from oracle import coarse as C
from paper_2406_00878_gb300 import workloads as W


def _edge_values(grid, fn, t):
    """Dirichlet data of one level (south nx, north nx, west ny, east ny) from fn(x, y, t)."""
    x = grid.xl + grid.hx * np.arange(1, grid.nx + 1)
    y = grid.yl + grid.hy * np.arange(1, grid.ny + 1)
    return np.concatenate([fn(x, grid.yl, t), fn(x, grid.yr, t), fn(grid.xl, y, t), fn(grid.xr, y, t)])


def _linear_heat(nx, ny, M, dt=0.01):
    # u = a + b x + c y + d t with constant mu: the 5-point Laplacian of u is zero and
    # BDF1 differentiates u exactly in t, so u is the discrete solution with q = d
    a, b, c, d = 0.3, -0.7, 1.1, 0.9
    fn = lambda x, y, t: a + b * np.asarray(x, dtype=float) + c * np.asarray(y, dtype=float) + d * t
    g = W.Grid(nx, ny, 0.0, 1.3, 0.2, 1.0)
    X, Y = g.nodes()
    u0 = fn(X, Y, 0.0).ravel()
    bc = np.array([_edge_values(g, fn, (n + 1) * dt) for n in range(M)])
    q = np.full((M, g.ns), d)
    exact = np.array([fn(X, Y, (n + 1) * dt).ravel() for n in range(M)])
    return W.Problem("linear_heat", g, W.Params(W.HEAT, 0.7, 0.0), M, dt, u0, bc, q), exact


def _linear_burgers(nx, ny, M, dt=0.02):
    # u = alpha(t) (1 + x + y), alpha linear in t: central differences of f = u^2/2 are exact
    # for quadratics, the viscous term vanishes, BDF1 is exact; q = (1 + x + y)(alpha' + 2 alpha^2)
    a0, a1 = 0.4, -0.6
    alpha = lambda t: a0 + a1 * t
    fn = lambda x, y, t: alpha(t) * (1.0 + np.asarray(x, dtype=float) + np.asarray(y, dtype=float))
    g = W.Grid(nx, ny)
    X, Y = g.nodes()
    u0 = fn(X, Y, 0.0).ravel()
    bc = np.array([_edge_values(g, fn, (n + 1) * dt) for n in range(M)])
    q = np.array([((1 + X + Y) * (a1 + 2 * alpha((n + 1) * dt) ** 2)).ravel() for n in range(M)])
    exact = np.array([fn(X, Y, (n + 1) * dt).ravel() for n in range(M)])
    return W.Problem("linear_burgers", g, W.Params(W.BURGERS, 0.05), M, dt, u0, bc, q), exact


@pytest.mark.parametrize("nx,ny,M,cf", [(15, 11, 8, 2), (14, 17, 10, 3), (31, 31, 16, 4), (20, 9, 7, 3)])
def test_linear_heat_solution_is_reproduced_exactly(nx, ny, M, cf):
    p, exact = _linear_heat(nx, ny, M)
    # the discrete solution of the fine problem is the linear function itself
    Uo, _ = oracle.sequential_bdf1(p.grid, p.params, M, p.dt, p.u0, p.bc, p.q)
    assert np.abs(Uo - exact).max() < 1e-12
    U, Uc, gc = C.coarse_guess(p.grid, p.params, M, p.dt, p.u0, p.bc, p.q, cf=cf)
    assert np.abs(U - exact).max() < 1e-12 * np.abs(exact).max()


@pytest.mark.parametrize("nx,M,cf", [(11, 6, 3), (15, 8, 4), (9, 4, 2)])
def test_linear_burgers_solution_is_reproduced_exactly(nx, M, cf):
    # M divisible by cf: the sources (quadratic in t) are sampled at coincident levels
    p, exact = _linear_burgers(nx, nx, M)
    U, Uc, gc = C.coarse_guess(p.grid, p.params, M, p.dt, p.u0, p.bc, p.q, cf=cf)
    assert np.abs(U - exact).max() < 1e-12 * np.abs(exact).max()


def test_restriction_is_injection_on_coincident_nodes():
    p = W.random_problem(3, 23, 17, 12, W.BURGERS, with_bc=True, with_q=True)
    cf = 3                              # 24 and 18 intervals, 12 levels: every third node and level
    gc, Mc, dtc, u0c, bcc, qc = C.restrict(p.grid, p.M, p.dt, p.u0, p.bc, p.q, cf)
    assert (gc.nx, gc.ny, Mc) == (7, 5, 4) and np.isclose(dtc, 3 * p.dt)
    fx = cf * np.arange(1, gc.nx + 1) - 1
    fy = cf * np.arange(1, gc.ny + 1) - 1
    u0 = p.u0.reshape(p.grid.ny, p.grid.nx)
    np.testing.assert_allclose(u0c.reshape(gc.ny, gc.nx), u0[np.ix_(fy, fx)], rtol=0, atol=1e-14)
    q = p.q.reshape(p.M, p.grid.ny, p.grid.nx)
    for l in range(Mc):
        lf = cf * (l + 1) - 1
        np.testing.assert_allclose(qc[l].reshape(gc.ny, gc.nx), q[lf][np.ix_(fy, fx)], rtol=0, atol=1e-14)
        b = p.bc[lf]
        nx, ny = p.grid.nx, p.grid.ny
        want = np.concatenate([b[:nx][fx], b[nx:2 * nx][fx], b[2 * nx:2 * nx + ny][fy], b[2 * nx + ny:][fy]])
        np.testing.assert_allclose(bcc[l], want, rtol=0, atol=1e-14)


def test_spline_stage_converges_at_fourth_order():
    # v = sin(pi t / T) sin(pi x) sin(2 pi y) on [0,1]^2 x [0,T] vanishes with its second
    # derivatives at every end, which is where natural splines are fourth-order accurate
    T, M, n = 0.5, 64, 63
    g = W.Grid(n, n)
    X, Y = g.nodes()
    v = lambda x, y, t: np.sin(np.pi * t / T) * np.sin(np.pi * x) * np.sin(2 * np.pi * y)
    exact = np.array([v(X, Y, (k + 1) * T / M).ravel() for k in range(M)])
    errs = []
    for cf in (4, 2):
        nxc, nyc, Mc = C.coarse_sizes(n, n, M, cf)
        gc = C._Grid(nxc, nyc, 0.0, 1.0, 0.0, 1.0)
        Xc, Yc = np.meshgrid(np.arange(1, nxc + 1) / (nxc + 1), np.arange(1, nyc + 1) / (nyc + 1), indexing="xy")
        Uc = np.array([v(Xc, Yc, (l + 1) * T / Mc).ravel() for l in range(Mc)])
        U = C.interpolate(g, M, T / M, np.zeros(g.ns), None, gc, Mc, Uc, None)
        errs.append(np.abs(U - exact).max())
    assert errs[1] < 1e-4 and errs[0] / errs[1] > 12.0, errs


def test_coarse_sizes_reject_too_small_grids():
    assert C.coarse_sizes(32, 32, 16, 4) == (7, 7, 4)
    assert C.coarse_sizes(62, 62, 12, 3) == (20, 20, 4)
    for args in [(2, 8, 8, 2), (8, 8, 1, 2), (8, 8, 8, 1)]:
        with pytest.raises(ValueError):
            C.coarse_sizes(*args)


def test_paper_guess_beats_the_plain_guess_on_heat():
    # the paper's heat setting coarsens by 4; the guess must start Newton much closer to
    # the solution (the noise in u^0 lives on no coarse grid, so the residual's max stays
    # of the same order) and save Newton iterations
    p = W.heat32(0)
    U, Uc, gc = C.coarse_guess(p.grid, p.params, p.M, p.dt, p.u0, p.bc, p.q, cf=4)
    Us, _ = oracle.sequential_bdf1(p.grid, p.params, p.M, p.dt, p.u0)
    e_plain, e_coarse = np.abs(p.plain_guess() - Us).max(), np.abs(U - Us).max()
    assert e_coarse < 0.25 * e_plain, (e_plain, e_coarse)
    Up, itp, _, _ = oracle.newton_all_at_once(p.grid, p.params, p.M, p.dt, p.u0, p.plain_guess(), tol=1e-13)
    Ug, itg, _, _ = oracle.newton_all_at_once(p.grid, p.params, p.M, p.dt, p.u0, U, tol=1e-13)
    assert 0 < itg < itp and np.abs(Ug - Up).max() < 1e-11
