"""Pins of the oracle's block inverse (eq. 6-8, Theorem 1) and level solvers.

* the nested block inverse equals a brute-force dense solve of eq. 6;
* it equals the decoupled product form of eq. 8 (Theorem 1), with and without
  the diagonal preconditioner of Sec. 7;
* Remark 2's diagonal count 2n^2 + 2n + 1 of P^n;
* eq. 15's bound N_t = 22 at N = 64, mu = 1e-3 (Sec. 7);
* constant-viscosity heat: A = I + tau mu L_h is diagonalised by the DST-I with
  the eigenvalues of eq. 14, a textbook solve to compare both level solvers with.
"""
import json
import os

import numpy as np
import pytest
import scipy.fft

import oracle
from paper_2406_00878_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _blocks(eq, nx, ny, M, seed):
    p = W.random_problem(seed, nx, ny, M, eq, with_bc=True)
    rng = np.random.default_rng(seed + 100)
    U = p.plain_guess() + 0.3 * rng.standard_normal((M, nx * ny))
    coef = oracle.jacobian(p.grid, p.params, M, p.dt * 20, U, p.bc)
    R = rng.standard_normal((M, nx * ny))
    return coef, R


@pytest.mark.parametrize("eq", [W.HEAT, W.BURGERS])
@pytest.mark.parametrize("solver", [oracle.SOLVER_BAND_LU, oracle.SOLVER_BICGSTAB])
def test_nested_inverse_equals_dense_global_solve(eq, solver):
    nx, ny, M = 4, 3, 5
    coef, R = _blocks(eq, nx, ny, M, 3)
    J = oracle.dense_global_jacobian(nx, ny, M, coef)
    dense = np.linalg.solve(J, R.ravel()).reshape(M, nx * ny)
    dU = oracle.block_solve(nx, ny, M, coef, R, solver=solver, rtol=1e-15)
    np.testing.assert_allclose(dU, dense, rtol=0, atol=1e-12 * np.abs(dense).max())
    # and it satisfies eq. 6 row by row: A_n du^n - du^{n-1} = r^n
    for n in range(M):
        lhs = oracle.apply_A(nx, ny, coef[:, n, :], dU[n]) - (dU[n - 1] if n else 0.0)
        np.testing.assert_allclose(lhs, R[n], rtol=0, atol=1e-12 * np.abs(R).max())


@pytest.mark.parametrize("eq", [W.HEAT, W.BURGERS])
@pytest.mark.parametrize("precondition", [False, True])
def test_product_form_theorem1_equals_nested_inverse(eq, precondition):
    nx, ny, M = 4, 4, 4
    coef, R = _blocks(eq, nx, ny, M, 5)
    dU = oracle.block_solve(nx, ny, M, coef, R, solver=oracle.SOLVER_BAND_LU)
    dV = oracle.product_form_solve(nx, ny, M, coef, R, diag_precondition=precondition)
    np.testing.assert_allclose(dV, dU, rtol=0, atol=1e-9 * np.abs(dU).max())


def test_remark2_diagonal_count():
    ref = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))["remark2"]
    nx = ny = 13
    M = max(ref["n"])
    coef, R = _blocks(W.BURGERS, nx, ny, M, 9)
    P, _ = oracle.product_form(nx, ny, M, coef, R[:M])
    for n, expect in zip(ref["n"], ref["diagonals"]):
        assert expect == 2 * n * n + 2 * n + 1
        assert oracle.nonzero_diagonals(P[n - 1], tol=1e-300) == expect


def test_eq15_largest_level_count():
    ref = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))["eq15"]
    assert oracle.max_levels_cond_bound(ref["N"], ref["mu"], ref["c"], ref["eps_rof"]) == ref["max_levels"]


@pytest.mark.parametrize("solver", [oracle.SOLVER_BAND_LU, oracle.SOLVER_BICGSTAB])
def test_constant_viscosity_block_matches_dst_diagonalisation(solver):
    nx, ny = 11, 7
    g = W.Grid(nx, ny, 0.0, 1.3, 0.0, 0.9)
    mu, dt = 0.6, 0.01
    rng = np.random.default_rng(2)
    u = rng.standard_normal(g.ns)  # the block does not depend on u when mu is constant
    cf = oracle.level_jacobian(g, W.Params(W.HEAT, mu, 0.0), dt, u)
    b = rng.standard_normal((ny, nx))
    kx = np.arange(1, nx + 1)
    ky = np.arange(1, ny + 1)
    lam_x = 4.0 / g.hx ** 2 * np.sin(np.pi * kx / (2 * (nx + 1))) ** 2
    lam_y = 4.0 / g.hy ** 2 * np.sin(np.pi * ky / (2 * (ny + 1))) ** 2
    lam = lam_y[:, None] + lam_x[None, :]
    x_dst = scipy.fft.idstn(scipy.fft.dstn(b, type=1) / (1.0 + dt * mu * lam), type=1)
    x = oracle.level_solve(nx, ny, cf, b.ravel(), solver=solver, rtol=1e-15)
    np.testing.assert_allclose(x, x_dst.ravel(), rtol=0, atol=1e-12 * np.abs(x_dst).max())
