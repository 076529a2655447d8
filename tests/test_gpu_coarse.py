"""f4: the paper's coarse-grid + cubic-spline initial iterate on the GPU against the
oracle (restriction, coarse sequential solve, natural splines along x, y, t).

Tolerance: both sides converge the coarse problem (the library to a tau-scaled residual
of 1e-13, the oracle's sequential BDF1 to 1e-14); the block system's inverse has norm
<= M_c for these problems, and the spline stage amplifies by less than 2 (the natural
spline's Lebesgue constant), so the guesses agree to 1e-10 of their size."""
import numpy as np
import pytest

import oracle
from oracle import coarse as C
from paper_2406_00878_gb300 import pit
from paper_2406_00878_gb300 import workloads as W
from tests import test_oracle_coarse as T

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _opt(tol=1e-13):
    o = pit.pit_default_options()
    o.tol_res = tol
    return o


def _gpu_guess(p, cf, opt=None):
    ctx = pit.context_for(p, opt or _opt())
    try:
        U = torch.empty((p.M, p.grid.ns), dtype=torch.float64, device="cuda")
        st, info = pit.pit_coarse_guess(ctx, cf, U.view(-1))
        return U.cpu().numpy(), info
    finally:
        ctx.close()


@pytest.mark.parametrize("seed,nx,ny,M,eq,cf,bc,q", [
    (0, 23, 17, 12, W.BURGERS, 3, True, True),     # coincident nodes and levels
    (1, 37, 23, 11, W.BURGERS, 3, True, True),     # ragged: nothing coincides in x, t
    (2, 30, 30, 16, W.HEAT, 4, False, False),
    (3, 45, 19, 9, W.HEAT, 2, True, False),
    (4, 64, 64, 24, W.BURGERS, 3, False, True),
])
def test_coarse_guess_matches_oracle(seed, nx, ny, M, eq, cf, bc, q):
    p = W.random_problem(seed, nx, ny, M, eq, with_bc=bc, with_q=q)
    U, info = _gpu_guess(p, cf)
    Uo, Uc, gc = C.coarse_guess(p.grid, p.params, M, p.dt, p.u0, p.bc, p.q, cf=cf)
    assert info["converged"]
    err = np.abs(U - Uo).max()
    assert err <= 1e-10 * np.abs(Uo).max(), err


@pytest.mark.parametrize("nx,ny,M,cf", [(15, 11, 8, 2), (20, 9, 7, 3), (31, 31, 16, 4)])
def test_linear_solution_is_reproduced_exactly(nx, ny, M, cf):
    p, exact = T._linear_heat(nx, ny, M)
    U, _ = _gpu_guess(p, cf)
    assert np.abs(U - exact).max() <= 1e-11 * np.abs(exact).max()


def test_newton_from_the_coarse_guess_reaches_the_same_solution():
    # heat32 coarsened by 4 (the paper's heat factor): the guess is much closer to the
    # solution than the plain guess, and Newton from it converges to the same solution in
    # no more iterations (inexact inner solves can make the counts equal)
    p = W.heat32(0)
    ctx = pit.context_for(p, _opt(1e-12))
    try:
        U = torch.empty((p.M, p.grid.ns), dtype=torch.float64, device="cuda")
        pit.pit_fill_plain_guess(ctx, U.view(-1))
        plain = U.clone()
        _, inf_plain = pit.pit_solve(ctx, U.view(-1))
        U_plain = U.clone()
        pit.pit_coarse_guess(ctx, 4, U.view(-1))
        guess = U.clone()
        _, inf_coarse = pit.pit_solve(ctx, U.view(-1))
    finally:
        ctx.close()
    assert inf_coarse["newton_iters"] <= inf_plain["newton_iters"], (inf_plain["newton_iters"], inf_coarse["newton_iters"])
    assert float((U - U_plain).abs().max()) <= 1e-10 * float(U_plain.abs().max())
    assert float((guess - U_plain).abs().max()) < 0.25 * float((plain - U_plain).abs().max())


def test_full_size_burgers256_guess_matches_oracle():
    # the smooth 256^2 x 256 Burgers workload coarsened by 3 (the paper's Burgers factor):
    # 84^2 nodes x 85 coarse levels; compared at every node
    p = W.burgers256(0)
    U, info = _gpu_guess(p, 3)
    Uo, _, _ = C.coarse_guess(p.grid, p.params, p.M, p.dt, p.u0, p.bc, p.q, cf=3)
    assert np.abs(U - Uo).max() <= 1e-10 * np.abs(Uo).max()


def test_invalid_factors_are_rejected():
    p = W.random_problem(5, 8, 8, 6, W.HEAT)
    ctx = pit.context_for(p)
    try:
        U = torch.empty((p.M, p.grid.ns), dtype=torch.float64, device="cuda")
        for cf in (1, 0, 5):            # cf = 5: (8 + 1) // 5 - 1 = 0 coarse nodes
            st, _ = pit.pit_coarse_guess(ctx, cf, U.view(-1), check=False)
            assert st == pit.PIT_EINVAL
    finally:
        ctx.close()


@pytest.mark.parametrize("nx,ny,M,cf", [(3, 5, 2, 2), (5, 5, 3, 3), (7, 4, 9, 2)])
def test_smallest_coarse_grids(nx, ny, M, cf):
    # one coarse node in a direction, a single coarse level, ragged sizes
    p = W.random_problem(40 + nx, nx, ny, M, W.BURGERS, with_bc=True, with_q=True)
    U, info = _gpu_guess(p, cf)
    Uo, _, _ = C.coarse_guess(p.grid, p.params, M, p.dt, p.u0, p.bc, p.q, cf=cf)
    assert np.abs(U - Uo).max() <= 1e-10 * np.abs(Uo).max()
