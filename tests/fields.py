"""Analytic fields for the pins: exact solutions, boundary sampling and
manufactured sources computed from the continuous PDE (eq. 1), never from the
discrete operator under test."""
import numpy as np

from paper_2406_00878_gb300 import workloads as W


def boundary(grid, fn, t):
    """Dirichlet data of fn(x, y, t) on one level in the layout south, north, west, east."""
    xs = grid.xl + grid.hx * np.arange(1, grid.nx + 1)
    ys = grid.yl + grid.hy * np.arange(1, grid.ny + 1)
    return np.concatenate([fn(xs, np.full_like(xs, grid.yl), t), fn(xs, np.full_like(xs, grid.yr), t),
                           fn(np.full_like(ys, grid.xl), ys, t), fn(np.full_like(ys, grid.xr), ys, t)])


def boundary_levels(grid, fn, M, dt):
    return np.ascontiguousarray(np.array([boundary(grid, fn, n * dt) for n in range(1, M + 1)]))


def on_nodes(grid, fn, t):
    X, Y = grid.nodes()
    return np.ascontiguousarray(fn(X, Y, t).ravel())


def continuous_F(params, u, ux, uy, uxx, uyy):
    """Continuous operator of eq. 1 (everything but u_t) from point values of u and
    its derivatives: f_x + g_y - (mu u_x)_x - (mu u_y)_y with f = g = beta u^2/2,
    mu = mu_a + mu_b u^2."""
    beta = 1.0 if params.equation == W.BURGERS else 0.0
    mu = params.mu_a + params.mu_b * u * u
    mup = 2.0 * params.mu_b * u
    return beta * u * (ux + uy) - mup * (ux * ux + uy * uy) - mu * (uxx + uyy)


class SteadyField:
    """u(x, y) = c0 sin(a x + 0.3) sin(b y + 0.7) + c1 x y with exact derivatives."""

    def __init__(self, c0=0.6, c1=0.4, a=2.1, b=1.7):
        self.c0, self.c1, self.a, self.b = c0, c1, a, b

    def u(self, x, y, t=0.0):
        return self.c0 * np.sin(self.a * x + 0.3) * np.sin(self.b * y + 0.7) + self.c1 * x * y

    def derivs(self, x, y):
        c0, c1, a, b = self.c0, self.c1, self.a, self.b
        sx, cx = np.sin(a * x + 0.3), np.cos(a * x + 0.3)
        sy, cy = np.sin(b * y + 0.7), np.cos(b * y + 0.7)
        u = c0 * sx * sy + c1 * x * y
        ux = c0 * a * cx * sy + c1 * y
        uy = c0 * b * sx * cy + c1 * x
        uxx = -c0 * a * a * sx * sy
        uyy = -c0 * b * b * sx * sy
        return u, ux, uy, uxx, uyy

    def source(self, params, grid):
        X, Y = grid.nodes()
        return np.ascontiguousarray(continuous_F(params, *self.derivs(X, Y)).ravel())
