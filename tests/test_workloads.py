"""The seeded synthetic inputs follow the recipes stated for them: sizes, parameters and
value laws of the headline, discontinuous, batched and learned-guess workloads, and the
same bytes for the same seed."""
import numpy as np

from paper_2406_00878_gb300 import workloads as W


def test_headline_and_discontinuous_workloads():
    p = W.burgers256()
    assert (p.grid.nx, p.grid.ny, p.M, p.dt) == (256, 256, 256, 1e-3) and p.dof == 16_777_216
    assert p.params == W.Params(W.BURGERS, 0.01, 0.0) and p.bc is None and p.q is None
    X, Y = p.grid.nodes()
    np.testing.assert_array_equal(p.u0, (np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y)).ravel())
    assert abs(X[0, 0] - 1.0 / 257) < 1e-15                      # interior nodes, h = 1/(nx + 1)
    q = W.burgers512(seed=3)
    assert (q.grid.nx, q.M, q.dt, q.params.mu_a) == (512, 1024, 5e-4, 1e-3)
    X, Y = q.grid.nodes()
    inside = (X >= 0.25) & (X <= 0.5) & (Y >= 0.25) & (Y <= 0.5)
    dev = q.u0.reshape(X.shape) - inside
    assert np.abs(dev).max() < 1e-2 and 0.8e-3 < dev.std() < 1.2e-3   # 1e-3 N(0, 1) noise
    np.testing.assert_array_equal(q.u0, W.burgers512(seed=3).u0)


def test_batched_workload_recipe():
    probs = W.batched(seed=0)
    assert len(probs) == 64
    for p in probs:
        assert p.grid.nx == p.grid.ny and p.grid.nx in range(64, 385, 32)
        assert p.M in range(32, 513, 32) and p.dt == 1e-3
        nu = p.meta["nu"]
        assert 1e-3 <= nu <= 1e-1
        if p.params.equation == W.HEAT:
            assert p.params.mu_a == nu and p.params.mu_b == nu        # mu = nu (1 + u^2)
        else:
            assert p.params == W.Params(W.BURGERS, nu, 0.0)
        u = p.u0.reshape(p.grid.ny, p.grid.nx)
        assert np.isfinite(u).all() and np.abs(u).max() > 0
    assert {p.params.equation for p in probs} == {W.HEAT, W.BURGERS}
    assert len({p.grid.nx for p in probs}) >= 8 and len({p.M for p in probs}) >= 8
    assert sum(p.dof for p in probs) == 1_019_314_176
    again = W.batched(seed=0)
    assert all(np.array_equal(a.u0, b.u0) and a.M == b.M for a, b in zip(probs, again))


def test_sine_series_vanishes_on_the_boundary_and_has_the_stated_spectrum():
    g = W.Grid(63, 63)
    rng = np.random.default_rng(7)
    u = W.fourier_u0(g, rng).reshape(63, 63)
    # the series of sin(k pi x) with k <= 8: extending the grid to the boundary nodes gives 0 there,
    # and a discrete sine transform of the interior values recovers only modes with kx^2 + ky^2 <= 64
    n = 64
    S = np.sin(np.pi * np.outer(np.arange(1, n), np.arange(1, n)) / n)
    A = S @ u @ S.T * (2.0 / n) ** 2
    kx, ky = np.meshgrid(np.arange(1, n), np.arange(1, n), indexing="ij")
    outside = (kx ** 2 + ky ** 2) > 64
    assert np.abs(A[outside]).max() < 1e-12 * np.abs(A).max()
    assert np.abs(A[~outside]).max() > 0.1
