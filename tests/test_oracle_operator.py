"""Pins of the oracle's discrete operator (eq. 3) and Jacobian blocks (eq. 5-6).

* closed forms: the 3-point central stencils are exact on low-degree
  polynomials, so the discrete F equals the continuous operator there;
* the paper's own printed errors (Table grconv_heat) reproduced digit for digit;
* finite differences of F against the analytic Jacobian;
* a manufactured steady solution converging at second order in space.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2406_00878_gb300 import workloads as W
from tests.fields import SteadyField, boundary, boundary_levels, continuous_F, on_nodes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _grid(nx=7, ny=5):
    return W.Grid(nx, ny, -0.3, 0.9, 0.2, 1.5)


def test_burgers_convection_exact_on_linear_fields():
    # f = u^2/2 is quadratic along a line when u is linear, so the central
    # difference (f_E - f_W)/(2h) is exact; the Laplacian of a linear u is 0.
    g = _grid()
    a, b, c = 0.7, -1.3, 0.45
    fn = lambda x, y, t: a + b * x + c * y
    params = W.Params(W.BURGERS, 0.37, 0.0)
    Fd = oracle.F(g, params, on_nodes(g, fn, 0.0), boundary(g, fn, 0.0))
    X, Y = g.nodes()
    u = fn(X, Y, 0).ravel()
    expect = u * (b + c)
    np.testing.assert_allclose(Fd, expect, rtol=1e-12, atol=1e-12)


def test_constant_viscosity_laplacian_exact_on_quadratics():
    g = _grid(6, 8)
    fn = lambda x, y, t: 0.3 + 0.2 * x - 0.5 * y + 1.1 * x * x - 0.7 * x * y + 0.9 * y * y
    for eq in (W.HEAT, W.BURGERS):
        params = W.Params(eq, 0.8, 0.0)
        Fd = oracle.F(g, params, on_nodes(g, fn, 0.0), boundary(g, fn, 0.0))
        X, Y = g.nodes()
        u = fn(X, Y, 0)
        ux = 0.2 + 2.2 * X - 0.7 * Y
        uy = -0.5 - 0.7 * X + 1.8 * Y
        if eq == W.HEAT:
            expect = continuous_F(params, u, ux, uy, 2.2, 1.8).ravel()
            np.testing.assert_allclose(Fd, expect, rtol=1e-11, atol=1e-11)
        else:
            # convection of a quadratic is not exact; check the viscous part alone
            Fv = Fd - oracle.F(g, W.Params(W.BURGERS, 0.0, 0.0), on_nodes(g, fn, 0.0), boundary(g, fn, 0.0))
            np.testing.assert_allclose(Fv, (-0.8 * (2.2 + 1.8)) * np.ones(g.ns), rtol=1e-11, atol=1e-11)


def test_nonlinear_viscosity_exact_on_linear_fields():
    # mu(u) = mu_a + mu_b u^2 with u linear: mu at the mid-point average is mu of
    # the exact mid-point value, and the flux difference is then exact:
    # -(mu u_x)_x - (mu u_y)_y = -mu'(u) (u_x^2 + u_y^2).
    g = _grid(9, 4)
    a, b, c = 1.5, 0.8, -0.6
    fn = lambda x, y, t: a + b * x + c * y
    params = W.Params(W.HEAT, 0.25, 0.7)
    Fd = oracle.F(g, params, on_nodes(g, fn, 0.0), boundary(g, fn, 0.0))
    X, Y = g.nodes()
    u = fn(X, Y, 0).ravel()
    np.testing.assert_allclose(Fd, -2 * 0.7 * u * (b * b + c * c), rtol=1e-11, atol=1e-12)


def test_residual_time_term_and_source():
    # with F = 0 (constant field, constant viscosity) the tau-scaled residual of eq. 5
    # is -(u^n - u^{n-1}) + tau q^n at every node
    g = _grid(4, 3)
    params = W.Params(W.HEAT, 1.3, 0.0)
    M, dt = 3, 0.1
    levels = [2.0, 2.5, 2.25, 3.0]
    u0 = np.full(g.ns, levels[0])
    U = np.array([np.full(g.ns, v) for v in levels[1:]])
    bc = np.array([np.full(2 * g.nx + 2 * g.ny, v) for v in levels[1:]])
    q = np.array([np.full(g.ns, s) for s in (1.0, -2.0, 0.5)])
    R = oracle.residual(g, params, M, dt, u0, U, bc, q)
    for n in range(M):
        np.testing.assert_allclose(R[n], -(levels[n + 1] - levels[n]) + dt * q[n, 0], rtol=0, atol=1e-14)


def test_paper_table_grconv_heat_reproduced():
    ref = json.load(open(os.path.join(GOLDEN, "grconv_heat.json")))
    mu0, alpha = 1e-6, 1.0
    exact = lambda x, y, t: np.sqrt(np.sqrt(alpha / mu0) * (x + y) + alpha * t + 1.0)
    errs = []
    for N in ref["N"]:
        g = W.Grid(N - 1, N - 1, 0.1, 1.1, 0.1, 1.1)
        M, dt = N, 1.0 / N
        p = W.Problem("heat_exact", g, W.Params(W.HEAT, 0.0, mu0), M, dt, on_nodes(g, exact, 0.0),
                      boundary_levels(g, exact, M, dt))
        U, it, res, _ = oracle.solve(p, tol=1e-12)
        err = max(np.abs(U[n - 1] - on_nodes(g, exact, n * dt)).max() for n in range(1, M + 1))
        errs.append(err)
    for err, printed in zip(errs, ref["linf_error"]):
        assert float(f"{err:.2e}") == pytest.approx(printed, rel=1e-9), (errs, ref["linf_error"])
    rates = [np.log(errs[k - 1] / errs[k]) / np.log(ref["N"][k] / ref["N"][k - 1]) for k in range(1, len(errs))]
    for r, printed in zip(rates, ref["linf_rate"][1:]):
        assert abs(r - printed) < 0.051, (rates, ref["linf_rate"])


@pytest.mark.parametrize("eq,mu_a,mu_b", [(W.HEAT, 0.4, 0.9), (W.HEAT, 0.0, 1.2), (W.BURGERS, 0.05, 0.0),
                                          (W.BURGERS, 0.05, 0.3)])
def test_jacobian_matches_finite_differences(eq, mu_a, mu_b):
    rng = np.random.default_rng(11)
    g = _grid(5, 4)
    params = W.Params(eq, mu_a, mu_b)
    dt = 0.37
    u = rng.uniform(-1.0, 1.5, g.ns)
    bnd = rng.uniform(-1.0, 1.0, 2 * g.nx + 2 * g.ny)
    cf = oracle.level_jacobian(g, params, dt, u, bnd)
    A = oracle.dense_block(g.nx, g.ny, cf)
    # central differences of u + dt F(u), column by column
    eps = 1e-6
    Afd = np.zeros_like(A)
    for k in range(g.ns):
        e = np.zeros(g.ns)
        e[k] = eps
        Afd[:, k] = ((u + e + dt * oracle.F(g, params, u + e, bnd)) -
                     (u - e + dt * oracle.F(g, params, u - e, bnd))) / (2 * eps)
    scale = np.abs(A).max()
    np.testing.assert_allclose(A, Afd, rtol=0, atol=1e-7 * scale)
    # the 5-point pattern: nothing outside the stencil
    assert np.all(np.abs(Afd[A == 0]) < 1e-7 * scale)


@pytest.mark.parametrize("eq,mu_a,mu_b", [(W.HEAT, 0.3, 0.5), (W.BURGERS, 0.1, 0.0)])
def test_manufactured_steady_solution_second_order_in_space(eq, mu_a, mu_b):
    # A steady u_s with source q = F_continuous(u_s): BDF1 is exact in time for a
    # steady state, so the error is the spatial one and must fall as h^2.
    field = SteadyField()
    params = W.Params(eq, mu_a, mu_b)
    errs, hs = [], []
    for n in (12, 24, 48):
        g = W.Grid(n, n, 0.0, 1.0, 0.0, 1.0)
        M, dt = 3, 0.05
        q = np.tile(field.source(params, g), (M, 1))
        p = W.Problem("mms", g, params, M, dt, on_nodes(g, field.u, 0.0), boundary_levels(g, field.u, M, dt), q)
        U, it, res, _ = oracle.solve(p, tol=1e-13)
        errs.append(np.abs(U - on_nodes(g, field.u, 0.0)[None, :]).max())
        hs.append(g.hx)
    orders = [np.log(errs[k - 1] / errs[k]) / np.log(hs[k - 1] / hs[k]) for k in (1, 2)]
    assert all(1.85 < o < 2.15 for o in orders), (errs, orders)
