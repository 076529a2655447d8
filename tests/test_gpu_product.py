"""f4: the literal product form of Theorem 1 (eq. 8) on the GPU -- the recursion of
Sec. 5 in diagonal-offset storage, diag(P^n) scaling, banded LU without pivoting --
against the oracle's dense product form and against the nested block inverse.

Tolerance: the scaled product system of level n has condition ~K^n (eq. 15); both
sides solve it with LU in FP64, so they agree to ~eps K^n. The cases below keep
K^M below 1e4 (small mu tau / h^2), where 1e-10 relative is a safe bound; one case past
the bound shows the loss of digits that the nested form avoids."""
import numpy as np
import pytest

import oracle
from paper_2406_00878_gb300 import pit
from paper_2406_00878_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def _iterate(p, seed, amp=0.1):
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(p.plain_guess() + amp * rng.standard_normal((p.M, p.grid.ns)))


def _gpu_product(p, U, R):
    with pit.context_for(p) as ctx:
        dU = torch.empty(p.dof, dtype=torch.float64, device="cuda")
        st, info = pit.pit_product_form_solve(ctx, _dev(U), _dev(R), dU)
        return dU.cpu().numpy().reshape(p.M, -1), info


@pytest.mark.parametrize("seed,nx,ny,M,eq", [(0, 4, 3, 3, W.HEAT), (1, 5, 5, 4, W.BURGERS), (2, 6, 4, 5, W.BURGERS),
                                             (3, 1, 6, 4, W.HEAT), (4, 6, 1, 3, W.BURGERS)])
def test_product_form_matches_dense_oracle(seed, nx, ny, M, eq):
    p = W.random_problem(seed, nx, ny, M, eq, with_bc=True, mu_a=0.02, mu_b=0.0, dt=1e-3)
    U = _iterate(p, seed)
    R = oracle.residual(p.grid, p.params, M, p.dt, p.u0, U, p.bc, p.q)
    coef = oracle.jacobian(p.grid, p.params, M, p.dt, U, p.bc)
    want = oracle.product_form_solve(nx, ny, M, coef, R, diag_precondition=True)
    got, info = _gpu_product(p, U, R)
    assert info["diagonals"] == 2 * M * M + 2 * M + 1 and info["half_band"] == M * nx
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()


@pytest.mark.parametrize("seed,n,M,eq", [(5, 15, 8, W.BURGERS), (6, 24, 12, W.HEAT), (7, 31, 6, W.BURGERS)])
def test_product_form_equals_nested_inverse(seed, n, M, eq):
    # Theorem 1: the decoupled systems have the same solution as eq. 6
    p = W.random_problem(seed, n, n + 3, M, eq, with_bc=True, with_q=True, mu_a=1e-3, mu_b=0.0, dt=1e-3)
    U = _iterate(p, seed)
    R = oracle.residual(p.grid, p.params, M, p.dt, p.u0, U, p.bc, p.q)
    coef = oracle.jacobian(p.grid, p.params, M, p.dt, U, p.bc)
    want = oracle.block_solve(n, n + 3, M, coef, R)
    got, info = _gpu_product(p, U, R)
    assert info["min_pivot"] > 0
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()


def test_newton_with_product_form_reaches_the_sequential_solution():
    p = W.burgers_shock()
    Us, _ = oracle.sequential_bdf1(p.grid, p.params, p.M, p.dt, p.u0, p.bc)
    with pit.context_for(p) as ctx:
        U = torch.empty(p.dof, dtype=torch.float64, device="cuda")
        pit.pit_fill_plain_guess(ctx, U)
        st, info = pit.pit_solve_product(ctx, U)
        Up = U.cpu().numpy().reshape(p.M, -1)
        # the nested-form solver from the same start reaches the same solution
        pit.pit_fill_plain_guess(ctx, U)
        pit.pit_solve(ctx, U)
        Un = U.cpu().numpy().reshape(p.M, -1)
    assert info["converged"] and info["res_inf"][-1] <= 1e-12
    assert np.abs(Up - Us).max() <= 1e-10 * np.abs(Us).max()
    assert np.abs(Un - Us).max() <= 1e-10 * np.abs(Us).max()


def test_product_form_loses_digits_past_the_condition_bound():
    # heat with mu ~ 1 on 32^2 and tau = 1/64: K ~ 1e2 per level (eq. 15), so P^8 has
    # condition ~1e16 -- the literal form's last level is wrong at O(1) while the nested
    # inverse (same exact solution, Theorem 1) stays exact
    p = W.heat32(0)
    M = 8
    p = W.truncated(p, M)
    U = p.plain_guess()
    R = oracle.residual(p.grid, p.params, M, p.dt, p.u0, U)
    coef = oracle.jacobian(p.grid, p.params, M, p.dt, U)
    want = oracle.block_solve(p.grid.nx, p.grid.ny, M, coef, R)
    got, info = _gpu_product(p, U, R)
    err = np.abs(got - want).max(axis=1) / np.abs(want).max()
    assert err[0] <= 1e-12                # level 1 is a plain A_1 solve
    assert not (err[-1] <= 1e-6), err     # the last level has lost many digits (or overflowed)


@pytest.mark.parametrize("seed,nx,ny,M", [(8, 7, 5, 1), (9, 1, 9, 3), (10, 9, 1, 4)])
def test_product_form_edge_shapes(seed, nx, ny, M):
    # M = 1 (P^1 = A_1: a plain level solve) and one-dimensional grids
    p = W.random_problem(seed, nx, ny, M, W.BURGERS, with_bc=True, mu_a=0.01, mu_b=0.0, dt=1e-3)
    U = _iterate(p, seed)
    R = oracle.residual(p.grid, p.params, M, p.dt, p.u0, U, p.bc, p.q)
    coef = oracle.jacobian(p.grid, p.params, M, p.dt, U, p.bc)
    want = oracle.block_solve(nx, ny, M, coef, R)
    got, info = _gpu_product(p, U, R)
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()


def test_newton_with_product_form_on_heat_with_sources():
    # heat with Dirichlet data and sources, within the conditioning bound (small mu tau / h^2)
    p = W.random_problem(12, 12, 10, 5, W.HEAT, with_bc=True, with_q=True, mu_a=0.05, mu_b=0.05, dt=1e-3)
    Us, _ = oracle.sequential_bdf1(p.grid, p.params, p.M, p.dt, p.u0, p.bc, p.q)
    with pit.context_for(p) as ctx:
        U = torch.empty(p.dof, dtype=torch.float64, device="cuda")
        pit.pit_fill_plain_guess(ctx, U)
        st, info = pit.pit_solve_product(ctx, U)
        Ug = U.cpu().numpy().reshape(p.M, -1)
    assert info["converged"]
    assert np.abs(Ug - Us).max() <= 1e-10 * np.abs(Us).max()
