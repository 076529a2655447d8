"""Seeded synthetic inputs for the all-at-once BDF1 solver.

This module only builds input data (grids, parameters, initial data u^0,
boundary data b, sources q) with numpy; it holds none of the method's
arithmetic.  Both the CUDA path and the CPU oracle receive byte-identical arrays
from here.

Problem shapes follow the paper's model problems (Sec. 2 and Sec. 8 of
arXiv 2406.00878: 2-D nonlinear heat and viscous Burgers on a uniform grid with
Dirichlet data) at the sizes this project benchmarks:

* ``heat32``      nonlinear heat, mu = 1 + u^2, 32 x 32 interior nodes on [0,1]^2,
                  u0 = sin(pi x) sin(pi y) + 0.01 N(0,1), dt = 1/64, M = 16;
* ``burgers256``  Burgers, nu = 0.01, 256 x 256 interior, u0 = sin(2 pi x) sin(2 pi y),
                  dt = 1e-3, M = 256;
* ``burgers512``  Burgers, nu = 1e-3, 512 x 512 interior, u0 = 1 on [0.25, 0.5]^2
                  plus 1e-3 N(0,1) on interior nodes, dt = 5e-4, M = 1024;
* ``random_problem`` small random problems (smooth + noisy u0, optional
                  boundary data and sources) for parity tests.

Grid convention: ``nx``, ``ny`` count interior nodes; node (j, i) sits at
x = xl + (i + 1) h_x, y = yl + (j + 1) h_y with h_x = (xr - xl)/(nx + 1).
Arrays are float64, x fastest: a level is ``[ny, nx]`` flattened, the space-time
iterate ``[M, ny, nx]`` flattened, boundary data ``[M, 2 nx + 2 ny]`` in the
order south row, north row, west column, east column.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

HEAT, BURGERS = 0, 1


@dataclass(frozen=True)
class Grid:
    nx: int
    ny: int
    xl: float = 0.0
    xr: float = 1.0
    yl: float = 0.0
    yr: float = 1.0

    @property
    def hx(self) -> float:
        return (self.xr - self.xl) / (self.nx + 1)

    @property
    def hy(self) -> float:
        return (self.yr - self.yl) / (self.ny + 1)

    @property
    def ns(self) -> int:
        return self.nx * self.ny

    def nodes(self):
        """Interior node coordinates as (X, Y), each shape (ny, nx)."""
        x = self.xl + self.hx * np.arange(1, self.nx + 1)
        y = self.yl + self.hy * np.arange(1, self.ny + 1)
        return np.meshgrid(x, y, indexing="xy")


@dataclass(frozen=True)
class Params:
    equation: int          # HEAT or BURGERS
    mu_a: float            # mu(u) = mu_a + mu_b u^2
    mu_b: float = 0.0


@dataclass
class Problem:
    name: str
    grid: Grid
    params: Params
    M: int
    dt: float
    u0: np.ndarray                      # (Ns,)
    bc: Optional[np.ndarray] = None     # (M, 2nx+2ny) or None = zero Dirichlet data
    q: Optional[np.ndarray] = None      # (M, Ns) or None = no source
    meta: dict = field(default_factory=dict)

    @property
    def dof(self) -> int:
        return self.M * self.grid.ns

    def plain_guess(self) -> np.ndarray:
        """The plain initial iterate u^n = u^0 for every level, shape (M, Ns)."""
        return np.tile(self.u0.reshape(1, -1), (self.M, 1))


def heat32(seed: int = 0) -> Problem:
    g = Grid(32, 32)
    X, Y = g.nodes()
    rng = np.random.default_rng(seed)
    u0 = np.sin(np.pi * X) * np.sin(np.pi * Y) + 0.01 * rng.standard_normal((g.ny, g.nx))
    return Problem("heat32", g, Params(HEAT, 1.0, 1.0), 16, 1.0 / 64.0, np.ascontiguousarray(u0.ravel()),
                   meta={"seed": seed})


def burgers256(seed: int = 0, M: int = 256) -> Problem:
    g = Grid(256, 256)
    X, Y = g.nodes()
    u0 = np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y)
    return Problem("burgers256", g, Params(BURGERS, 0.01), M, 1e-3, np.ascontiguousarray(u0.ravel()),
                   meta={"seed": seed})


def burgers512(seed: int = 0, M: int = 1024) -> Problem:
    g = Grid(512, 512)
    X, Y = g.nodes()
    rng = np.random.default_rng(seed)
    box = ((X >= 0.25) & (X <= 0.5) & (Y >= 0.25) & (Y <= 0.5)).astype(np.float64)
    u0 = box + 1e-3 * rng.standard_normal((g.ny, g.nx))
    return Problem("burgers512", g, Params(BURGERS, 1e-3), M, 5e-4, np.ascontiguousarray(u0.ravel()),
                   meta={"seed": seed})


def burgers_shock(n: int = 63, M: int = 12, nu: float = 1e-3, v: float = 0.5, seed: int = 0) -> Problem:
    """The paper's Burgers test (Sec. 8.2): the viscous shock u = v/2 (1 - tanh(v (x + y - v t) / (4 nu)))
    on [0,1]^2 (domain: a reading), n x n interior nodes, M levels over T = 1, initial and Dirichlet
    data from the exact solution (63^2 x 12 is the setting of the paper's Newton-history figure)."""
    g = Grid(n, n)
    dt = 1.0 / M
    ex = lambda x, y, t: 0.5 * v * (1.0 - np.tanh(v * (x + y - v * t) / (4 * nu)))
    X, Y = g.nodes()
    x = g.hx * np.arange(1, n + 1)
    bc = np.array([np.concatenate([ex(x, 0.0, t), ex(x, 1.0, t), ex(0.0, x, t), ex(1.0, x, t)])
                   for t in dt * np.arange(1, M + 1)])
    return Problem(f"burgers_shock{n}x{M}", g, Params(BURGERS, nu), M, dt, np.ascontiguousarray(ex(X, Y, 0.0).ravel()),
                   np.ascontiguousarray(bc), meta={"seed": seed})


def by_name(name: str, seed: int = 0, **kw) -> Problem:
    return {"heat32": heat32, "burgers256": burgers256, "burgers512": burgers512,
            "burgers_shock": burgers_shock}[name](seed=seed, **kw)


def truncated(problem: Problem, M: int) -> Problem:
    """The same problem restricted to its first M levels. Because the all-at-once
    system is block lower-triangular in time, its solution equals the first M
    levels of the full solution."""
    return Problem(problem.name + f"[:{M}]", problem.grid, problem.params, M, problem.dt, problem.u0,
                   None if problem.bc is None else np.ascontiguousarray(problem.bc[:M]),
                   None if problem.q is None else np.ascontiguousarray(problem.q[:M]), dict(problem.meta))


def random_problem(seed: int, nx: int, ny: int, M: int, equation: int, with_bc: bool = False,
                   with_q: bool = False, amp: float = 1.0, dt: Optional[float] = None,
                   mu_a: Optional[float] = None, mu_b: Optional[float] = None) -> Problem:
    """A small random problem: smooth sine data plus noise, optional Dirichlet data and source."""
    rng = np.random.default_rng(seed)
    g = Grid(nx, ny, 0.0, float(rng.uniform(0.8, 1.2)), 0.0, float(rng.uniform(0.8, 1.2)))
    X, Y = g.nodes()
    kx, ky = rng.integers(1, 4, size=2)
    u0 = amp * (np.sin(kx * np.pi * X / g.xr) * np.sin(ky * np.pi * Y / g.yr) + 0.05 * rng.standard_normal(X.shape))
    if equation == HEAT:
        params = Params(HEAT, 0.5 if mu_a is None else mu_a, 0.5 if mu_b is None else mu_b)
        dt = 2e-3 if dt is None else dt
    else:
        params = Params(BURGERS, 0.02 if mu_a is None else mu_a, 0.0 if mu_b is None else mu_b)
        dt = 2e-3 if dt is None else dt
    bc = None
    if with_bc:
        bc = np.ascontiguousarray(0.2 * amp * rng.standard_normal((M, 2 * nx + 2 * ny)))
    q = None
    if with_q:
        q = np.ascontiguousarray(0.5 * amp * rng.standard_normal((M, g.ns)))
    return Problem(f"rand{seed}_{nx}x{ny}x{M}_{'heat' if equation == HEAT else 'burgers'}", g, params, M, dt,
                   np.ascontiguousarray(u0.ravel()), bc, q, meta={"seed": seed})


def fourier_u0(grid: Grid, rng, kmax: int = 8) -> np.ndarray:
    """u0 = sum over kx, ky >= 1 with kx^2 + ky^2 <= kmax^2 of a_k sin(kx pi x') sin(ky pi y'),
    a_k ~ N(0, 1/(kx^2 + ky^2)), x' = (x - xl)/(xr - xl): a random smooth field that
    vanishes on the boundary (zero Dirichlet data)."""
    X, Y = grid.nodes()
    xs = (X - grid.xl) / (grid.xr - grid.xl)
    ys = (Y - grid.yl) / (grid.yr - grid.yl)
    u = np.zeros_like(X)
    for kx in range(1, kmax + 1):
        for ky in range(1, kmax + 1):
            k2 = kx * kx + ky * ky
            if k2 > kmax * kmax:
                continue
            u += rng.normal(0.0, 1.0 / np.sqrt(k2)) * np.sin(kx * np.pi * xs) * np.sin(ky * np.pi * ys)
    return np.ascontiguousarray(u.ravel())


def batched(seed: int = 0, count: int = 64, sizes=tuple(range(64, 385, 32)), levels=tuple(range(32, 513, 32)),
            dt: float = 1e-3):
    """Independent problems of uneven size: square grids drawn from `sizes` (interior
    nodes), M from `levels`, nu log-uniform in [1e-3, 1e-1], Burgers or heat by a coin
    flip (heat: mu = nu (1 + u^2)), u0 a random sine series with modes k <= 8."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(sizes))
        M = int(rng.choice(levels))
        nu = float(10.0 ** rng.uniform(-3.0, -1.0))
        heat = bool(rng.integers(0, 2))
        g = Grid(n, n)
        params = Params(HEAT, nu, nu) if heat else Params(BURGERS, nu, 0.0)
        out.append(Problem(f"batch{seed}_{i}_{'heat' if heat else 'burgers'}{n}x{M}", g, params, M, dt,
                           fourier_u0(g, rng), meta={"seed": seed, "index": i, "nu": nu}))
    return out
