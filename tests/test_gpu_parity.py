"""GPU parity: every row of the hot path through the C ABI against the FP64 oracle
on the same seeded inputs.

Tolerances (FP64 on both sides, different association of the same formulas):
  (a1) residual:  |dr| <= 1e-14 * S, S the magnitude of the largest term of eq. 5
                  at that size (|u| plus the tau-scaled flux terms);
  (a2) Jacobian:  |dA| <= 1e-14 * max|A| per plane;
  (a3) block solve with eta = 1e-14: |ddU| <= 1e-10 * max|dU|;
  (a4) converged solution: max|U - U_oracle| <= 1e-10 * max|U_oracle|.
"""
import numpy as np
import pytest

import oracle
from paper_2406_00878_gb300 import pit
from paper_2406_00878_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def _term_scale(p, U):
    """Largest magnitude among the terms that enter the residual of eq. 5."""
    g = p.grid
    umax = max(np.abs(U).max(), np.abs(p.u0).max(), 1e-300)
    if p.bc is not None:
        umax = max(umax, np.abs(p.bc).max())
    mu = p.params.mu_a + p.params.mu_b * umax ** 2
    visc = 4 * p.dt * (1 / g.hx ** 2 + 1 / g.hy ** 2) * mu * umax * (1 + 2 * p.params.mu_b * umax ** 2 / max(mu, 1e-300))
    conv = (p.dt * (1 / g.hx + 1 / g.hy) * umax ** 2) if p.params.equation == W.BURGERS else 0.0
    q = p.dt * np.abs(p.q).max() if p.q is not None else 0.0
    return umax + visc + conv + q


def _perturbed_iterate(p, seed, amp=0.2):
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(p.plain_guess() + amp * rng.standard_normal((p.M, p.grid.ns)))


CASES = [
    # (seed, nx, ny, M, equation, bc, q, mu_b override)
    (1, 1, 1, 1, W.HEAT, False, False, None),
    (2, 3, 5, 2, W.BURGERS, True, True, None),
    (3, 17, 33, 3, W.HEAT, True, False, None),
    (4, 33, 17, 4, W.BURGERS, False, True, None),
    (5, 64, 48, 2, W.BURGERS, True, True, 0.4),
    (6, 1, 37, 3, W.HEAT, True, True, None),
    (7, 41, 1, 3, W.BURGERS, True, False, None),
    (8, 130, 97, 2, W.HEAT, False, False, 0.0),
]


def _case(c):
    seed, nx, ny, M, eq, bc, q, mub = c
    return W.random_problem(seed, nx, ny, M, eq, with_bc=bc, with_q=q, mu_b=mub)


@pytest.mark.parametrize("case", CASES, ids=[f"{c[1]}x{c[2]}x{c[3]}-{c[4]}" for c in CASES])
def test_residual_matches_oracle(case):
    p = _case(case)
    U = _perturbed_iterate(p, case[0] + 50)
    with pit.context_for(p) as ctx:
        R = torch.empty(p.M * p.grid.ns, dtype=torch.float64, device="cuda")
        rinf = pit.pit_residual(ctx, _dev(U), R)
        Rg = R.cpu().numpy().reshape(p.M, -1)
    Ro = oracle.residual(p.grid, p.params, p.M, p.dt, p.u0, U, p.bc, p.q)
    atol = 1e-14 * _term_scale(p, U)
    np.testing.assert_allclose(Rg, Ro, rtol=0, atol=atol)
    assert rinf == np.abs(Rg).max()


@pytest.mark.parametrize("case", CASES, ids=[f"{c[1]}x{c[2]}x{c[3]}-{c[4]}" for c in CASES])
def test_jacobian_matches_oracle(case):
    p = _case(case)
    U = _perturbed_iterate(p, case[0] + 60)
    with pit.context_for(p) as ctx:
        coef = torch.empty(5 * p.M * p.grid.ns, dtype=torch.float64, device="cuda")
        pit.pit_assemble(ctx, _dev(U), coef)
        cg = coef.cpu().numpy().reshape(5, p.M, -1)
    co = oracle.jacobian(p.grid, p.params, p.M, p.dt, U, p.bc)
    for c in range(5):
        np.testing.assert_allclose(cg[c], co[c], rtol=0, atol=1e-14 * max(np.abs(co[c]).max(), 1.0))


@pytest.mark.parametrize("solver", [pit.PIT_LIN_AUTO, pit.PIT_LIN_SOR, pit.PIT_LIN_BICGSTAB])
@pytest.mark.parametrize("case,team", [(CASES[2], 0), (CASES[2], 5), (CASES[3], 3), (CASES[4], 0), (CASES[4], 7),
                                       (CASES[5], 4), (CASES[6], 1), (CASES[7], 0), (CASES[7], 9)])
def test_block_solve_matches_oracle(case, team, solver):
    p = _case(case)
    U = _perturbed_iterate(p, case[0] + 70, amp=0.05)
    rng = np.random.default_rng(case[0] + 80)
    R = rng.standard_normal((p.M, p.grid.ns))
    opt = pit.pit_default_options()
    opt.team_ctas = team
    opt.lin_solver = solver
    opt.lin_max_iter = 20000
    with pit.context_for(p, opt) as ctx:
        dU = torch.empty(p.M * p.grid.ns, dtype=torch.float64, device="cuda")
        info = pit.pit_block_solve(ctx, _dev(U), _dev(R), dU, eta=1e-14)
        dg = dU.cpu().numpy().reshape(p.M, -1)
    coef = oracle.jacobian(p.grid, p.params, p.M, p.dt, U, p.bc)
    do = oracle.block_solve(p.grid.nx, p.grid.ny, p.M, coef, R, solver=oracle.SOLVER_BAND_LU)
    np.testing.assert_allclose(dg, do, rtol=0, atol=1e-10 * np.abs(do).max())
    assert info["levels_capped"] == 0


SOLVE_CASES = [
    lambda: W.heat32(0),
    lambda: W.heat32(3),
    lambda: W.random_problem(11, 23, 19, 5, W.BURGERS, with_bc=True, with_q=True),
    lambda: W.random_problem(12, 16, 31, 6, W.HEAT, with_bc=True, with_q=True),
    lambda: W.truncated(W.burgers256(0), 4),
    lambda: W.truncated(W.burgers512(0), 2),
]


@pytest.mark.parametrize("make", SOLVE_CASES, ids=["heat32s0", "heat32s3", "burg23x19", "heat16x31", "b256[:4]",
                                                   "b512[:2]"])
def test_newton_solve_matches_oracle(make):
    p = make()
    Uo, it_o, res_o, _ = oracle.solve(p, tol=1e-13)
    with pit.context_for(p) as ctx:
        U = torch.empty(p.dof, dtype=torch.float64, device="cuda")
        pit.pit_fill_plain_guess(ctx, U)
        status, info = pit.pit_solve(ctx, U)
        Ug = U.cpu().numpy().reshape(p.M, -1)
    assert info["converged"] and info["res_inf"][-1] <= 1e-12
    assert np.abs(Ug - Uo).max() <= 1e-10 * np.abs(Uo).max()
    # the GPU iterate satisfies the oracle's discrete system (eq. 4) to the tolerance
    Rchk = oracle.residual(p.grid, p.params, p.M, p.dt, p.u0, Ug, p.bc, p.q)
    assert np.abs(Rchk).max() <= 2e-12


def test_newton_step_matches_oracle_step():
    p = W.random_problem(13, 20, 14, 4, W.BURGERS, with_bc=True)
    opt = pit.pit_default_options()
    opt.eta_max = 1e-14  # a nearly exact Newton step
    opt.eta_gamma = 0.0
    U0 = p.plain_guess()
    Uo, _, _, _ = oracle.newton_all_at_once(p.grid, p.params, p.M, p.dt, p.u0, U0, p.bc, p.q, tol=0.0, maxit=1)
    with pit.context_for(p, opt) as ctx:
        U = _dev(U0)
        info = pit.pit_newton_step(ctx, U)
        Ug = U.cpu().numpy().reshape(p.M, -1)
    np.testing.assert_allclose(Ug, Uo, rtol=0, atol=1e-11 * np.abs(Uo).max())
    assert info["upd_rms"] > 0


def test_solve_host_equals_device_solve():
    p = W.random_problem(14, 24, 20, 5, W.HEAT, with_bc=True)
    with pit.context_for(p) as ctx:
        U = torch.empty(p.dof, dtype=torch.float64, device="cuda")
        pit.pit_fill_plain_guess(ctx, U)
        pit.pit_solve(ctx, U)
        Ud = U.cpu().numpy()
        Uh = np.zeros(p.dof)
        pit.pit_solve_host(ctx, np.ascontiguousarray(p.u0), Uh)
    np.testing.assert_array_equal(Uh, Ud)


def test_full_size_burgers256_sampled_levels_and_residual_property():
    # The bench workload itself (256 x 256, M = 256). The all-at-once system is block
    # lower-triangular in time, so the oracle can compute the first levels alone; the
    # residual of the whole GPU solution is checked by the oracle at every level.
    p = W.burgers256(0)
    with pit.context_for(p) as ctx:
        U = torch.empty(p.dof, dtype=torch.float64, device="cuda")
        pit.pit_fill_plain_guess(ctx, U)
        status, info = pit.pit_solve(ctx, U)
        Ug = U.cpu().numpy().reshape(p.M, -1)
    assert info["converged"]
    L = 6
    Uo, _, _, _ = oracle.solve(W.truncated(p, L), tol=1e-13)
    assert np.abs(Ug[:L] - Uo).max() <= 1e-10 * np.abs(Uo).max()
    Rchk = oracle.residual(p.grid, p.params, p.M, p.dt, p.u0, Ug)
    assert np.abs(Rchk).max() <= 2e-12


def test_errors_are_reported():
    p = W.random_problem(15, 12, 12, 3, W.HEAT)
    opt = pit.pit_default_options()
    opt.newton_max = 1
    with pit.context_for(p, opt) as ctx:
        U = torch.empty(p.dof, dtype=torch.float64, device="cuda")
        pit.pit_fill_plain_guess(ctx, U)
        status, info = pit.pit_solve(ctx, U, check=False)
        assert status == pit.PIT_ENOCONV and info["newton_iters"] == 1 and not info["converged"]
        # the last iterate is kept: it equals one Newton step from the plain guess
        assert torch.isfinite(U).all()
    bad = W.random_problem(15, 12, 12, 3, W.HEAT)
    bad.u0 = bad.u0.copy()
    bad.u0[5] = np.nan
    with pit.context_for(bad) as ctx:
        U = torch.empty(bad.dof, dtype=torch.float64, device="cuda")
        pit.pit_fill_plain_guess(ctx, U)
        status, info = pit.pit_solve(ctx, U, check=False)
        assert status == pit.PIT_EDIVERGED
        with pytest.raises(pit.PitError):
            pit.pit_residual(ctx, U, U)


def test_device_wait_timeout_is_reported_and_the_device_stays_usable():
    # a wait budget of one poll: the first team wait that is not satisfied at once gives up,
    # raises the abort flag for the other CTAs and the launch ends with PIT_ETIMEOUT (no
    # fault, no hang); a fresh context on the same device then solves normally
    p = W.random_problem(16, 64, 48, 4, W.BURGERS, with_bc=True)
    for teams in (-1, 0):                       # per-stage launches (chain kernel) and the wavefront
        opt = pit.pit_default_options()
        opt.wait_budget = 1
        opt.team_ctas = 8
        opt.wave_teams = teams
        with pit.context_for(p, opt) as ctx:
            U = torch.empty(p.dof, dtype=torch.float64, device="cuda")
            pit.pit_fill_plain_guess(ctx, U)
            status, info = pit.pit_solve(ctx, U, check=False)
            assert status == pit.PIT_ETIMEOUT, status
            assert "budget" in pit.lib().pit_last_error(ctx.handle).decode()
    Uo, _, _, _ = oracle.solve(p, tol=1e-13)
    with pit.context_for(p) as ctx:
        U = torch.empty(p.dof, dtype=torch.float64, device="cuda")
        pit.pit_fill_plain_guess(ctx, U)
        status, info = pit.pit_solve(ctx, U)
        assert info["converged"]
        assert np.abs(U.cpu().numpy().reshape(p.M, -1) - Uo).max() <= 1e-10 * np.abs(Uo).max()


WAVE_CASES = [
    (lambda: W.heat32(1), "heat32s1"),
    (lambda: W.random_problem(31, 37, 45, 7, W.BURGERS, with_bc=True, with_q=True), "burg37x45"),
    (lambda: W.random_problem(32, 20, 26, 9, W.HEAT, with_bc=True, with_q=True, mu_b=0.0), "linheat20x26"),
]


@pytest.mark.parametrize("teams", [-1, 1, 2, 3, 4, 6])
@pytest.mark.parametrize("make,name", WAVE_CASES, ids=[c[1] for c in WAVE_CASES])
def test_wavefront_solve_matches_oracle(make, name, teams):
    p = make()
    Uo, _, _, _ = oracle.solve(p, tol=1e-13)
    opt = pit.pit_default_options()
    opt.wave_teams = teams
    with pit.context_for(p, opt) as ctx:
        U = torch.empty(p.dof, dtype=torch.float64, device="cuda")
        pit.pit_fill_plain_guess(ctx, U)
        status, info = pit.pit_solve(ctx, U)
        Ug = U.cpu().numpy().reshape(p.M, -1)
    assert info["converged"] and info["res_inf"][-1] <= 1e-12
    if teams >= 1:
        assert info["wave_teams"] >= 1 and info["wave_launches"] >= 1
    assert np.abs(Ug - Uo).max() <= 1e-10 * np.abs(Uo).max()


def test_wavefront_iterates_equal_classic_newton_iterates():
    # with exact level solves the wavefront runs the same Newton iterates as the
    # per-stage launches: compare after a fixed number of iterations
    p = W.random_problem(33, 30, 22, 6, W.BURGERS, with_bc=True)
    outs = []
    for teams in (-1, 3):
        opt = pit.pit_default_options()
        opt.wave_teams = teams
        opt.newton_max = 2
        opt.eta_max = 1e-14
        opt.eta_gamma = 0.0
        with pit.context_for(p, opt) as ctx:
            U = torch.empty(p.dof, dtype=torch.float64, device="cuda")
            pit.pit_fill_plain_guess(ctx, U)
            pit.pit_solve(ctx, U, check=False)
            outs.append(U.cpu().numpy())
    np.testing.assert_allclose(outs[1], outs[0], rtol=0, atol=1e-11 * np.abs(outs[0]).max())


@pytest.mark.parametrize("prec", [pit.PIT_FP64, pit.PIT_FP32_INNER])
def test_wavefront_teams_of_different_sizes_run_the_same_iterates(prec):
    # The SMs that equal teams leave over go to the middle teams (shorter strips), and each
    # CTA then waits on the predecessor team's CTAs that own its rows. 64 x 256 interior
    # nodes: six teams of 24 CTAs (11-row strips) leave 8 of 152 SMs, which give four teams
    # 26 CTAs (10-row strips). The iterates must be those of equal teams bit for bit (the
    # red-black sweeps and the max-reductions do not depend on the strips), and the oracle's.
    p = W.random_problem(5, 64, 256, 8, W.BURGERS, with_bc=True)
    outs, infos = [], []
    for fixed in (False, True):
        opt = pit.pit_default_options()
        opt.precision = prec
        if fixed:
            opt.team_ctas = infos[0]["wave_team_ctas"]
        with pit.context_for(p, opt) as ctx:
            U = torch.empty(p.dof, dtype=torch.float64, device="cuda")
            pit.pit_fill_plain_guess(ctx, U)
            status, info = pit.pit_solve(ctx, U)
            outs.append(U.cpu().numpy())
            infos.append(info)
    auto, equal = infos
    assert auto["converged"] and equal["converged"]
    assert equal["wave_ctas"] == equal["wave_teams"] * equal["wave_team_ctas"]
    if torch.cuda.get_device_properties(0).multi_processor_count == 152:
        assert auto["wave_ctas"] > auto["wave_teams"] * auto["wave_team_ctas"]
    assert auto["wave_ctas"] <= torch.cuda.get_device_properties(0).multi_processor_count
    assert np.array_equal(outs[0], outs[1])
    Uo, _, _, _ = oracle.solve(p, tol=1e-13)
    assert np.abs(outs[0].reshape(p.M, -1) - Uo).max() <= 1e-10 * np.abs(Uo).max()


def _window_residual(p, U, start, count):
    """Oracle residual of levels start..start+count-1 of U (level n depends only on U[n-1], U[n])."""
    u_prev = p.u0 if start == 0 else U[start - 1]
    sub = W.Problem("window", p.grid, p.params, count, p.dt, np.ascontiguousarray(u_prev),
                    None if p.bc is None else np.ascontiguousarray(p.bc[start:start + count]),
                    None if p.q is None else np.ascontiguousarray(p.q[start:start + count]))
    return oracle.residual(sub.grid, sub.params, count, sub.dt, sub.u0, U[start:start + count], sub.bc, sub.q)


MIXED_CASES = [
    (lambda: W.heat32(2), "heat32s2"),
    (lambda: W.random_problem(41, 33, 29, 6, W.BURGERS, with_bc=True, with_q=True), "burg33x29"),
    (lambda: W.truncated(W.burgers256(0), 4), "b256[:4]"),
    (lambda: W.truncated(W.burgers512(0), 2), "b512[:2]"),
]


@pytest.mark.parametrize("make,name", MIXED_CASES, ids=[c[1] for c in MIXED_CASES])
def test_fp32_inner_solves_reach_the_fp64_solution(make, name):
    # f1: level solves in FP32 inside FP64 Newton; the converged iterate must still
    # satisfy the FP64 system to 1e-12 and match the FP64 oracle to 1e-10
    p = make()
    Uo, _, _, _ = oracle.solve(p, tol=1e-13)
    opt = pit.pit_default_options()
    opt.precision = pit.PIT_FP32_INNER
    with pit.context_for(p, opt) as ctx:
        U = torch.empty(p.dof, dtype=torch.float64, device="cuda")
        pit.pit_fill_plain_guess(ctx, U)
        status, info = pit.pit_solve(ctx, U)
        Ug = U.cpu().numpy().reshape(p.M, -1)
    assert info["converged"] and info["res_inf"][-1] <= 1e-12
    assert np.abs(Ug - Uo).max() <= 1e-10 * np.abs(Uo).max()


def test_fp32_inner_full_size_burgers512():
    # the mixed-precision workload at full size (512 x 512, M = 1024, windows of 32
    # levels, the launch configuration the benchmark times): the first levels against
    # the oracle's solution, the oracle's residual of the GPU solution at EVERY level
    # (268 M unknowns; the all-at-once system has a bounded inverse, so a residual at
    # round-off certifies the solution), and the whole solution against the FP64 GPU
    # solve of the same problem
    import os
    p = W.burgers512(0)
    sols = {}
    for prec in (pit.PIT_FP32_INNER, pit.PIT_FP64):
        opt = pit.pit_default_options()
        opt.precision = prec
        opt.window = 32
        with pit.context_for(p, opt) as ctx:
            U = torch.empty(p.dof, dtype=torch.float64, device="cuda")
            pit.pit_fill_plain_guess(ctx, U)
            status, info = pit.pit_solve(ctx, U)
            assert info["converged"]
            sols[prec] = U.cpu().numpy().reshape(p.M, -1)
    Ug = sols[pit.PIT_FP32_INNER]
    Uo, _, _, _ = oracle.solve(W.truncated(p, 2), tol=1e-13)
    assert np.abs(Ug[:2] - Uo).max() <= 1e-10 * np.abs(Uo).max()
    oracle.use_threads(len(os.sched_getaffinity(0)))   # bitwise the single-threaded oracle
    try:
        R = oracle.residual(p.grid, p.params, p.M, p.dt, p.u0, Ug)
    finally:
        oracle.use_threads(1)
    assert np.isfinite(R).all() and np.abs(R).max() <= 2e-12
    del R
    U64 = sols[pit.PIT_FP64]
    assert np.abs(Ug - U64).max() <= 1e-10 * np.abs(U64).max()


@pytest.mark.parametrize("window,teams,prec", [(1, 0, 0), (3, 2, 0), (4, 0, 1), (7, 3, 1)])
def test_windowed_solve_matches_oracle(window, teams, prec):
    # the all-at-once system is block lower-triangular in time: solving it window by
    # window gives the same solution
    p = W.random_problem(51, 27, 31, 9, W.BURGERS, with_bc=True, with_q=True)
    Uo, _, _, _ = oracle.solve(p, tol=1e-13)
    opt = pit.pit_default_options()
    opt.window, opt.wave_teams, opt.precision = window, teams, prec
    with pit.context_for(p, opt) as ctx:
        U = torch.empty(p.dof, dtype=torch.float64, device="cuda")
        pit.pit_fill_plain_guess(ctx, U)
        status, info = pit.pit_solve(ctx, U)
        Ug = U.cpu().numpy().reshape(p.M, -1)
    assert info["converged"] and info["windows"] == -(-p.M // window)
    assert np.abs(Ug - Uo).max() <= 1e-10 * np.abs(Uo).max()


def test_a_smaller_context_does_not_break_a_larger_one():
    # kernel launch limits are per kernel, not per context: creating a context for a
    # small grid after a large one must leave the large one's launches valid
    big = W.random_problem(21, 96, 96, 6, W.BURGERS)
    small = W.random_problem(22, 6, 6, 3, W.HEAT)
    Uo, _, _, _ = oracle.solve(big, tol=1e-13)
    with pit.context_for(big) as cb:
        with pit.context_for(small) as cs:
            Us = torch.empty(small.dof, dtype=torch.float64, device="cuda")
            pit.pit_fill_plain_guess(cs, Us)
            pit.pit_solve(cs, Us)
        U = torch.empty(big.dof, dtype=torch.float64, device="cuda")
        pit.pit_fill_plain_guess(cb, U)
        status, info = pit.pit_solve(cb, U)
    assert info["converged"]
    assert np.abs(U.cpu().numpy().reshape(big.M, -1) - Uo).max() <= 1e-10 * np.abs(Uo).max()


def test_windowed_solve_starts_from_the_given_iterate():
    # pit_solve with windows and PIT_START_GIVEN: a near-solution start saves Newton
    # updates; a wild start diverges in its window, which restarts from the plain guess;
    # both reach the oracle's solution
    p = W.random_problem(52, 27, 31, 9, W.BURGERS, with_bc=True, with_q=True)
    Uo, _, _, _ = oracle.solve(p, tol=1e-13)
    opt = pit.pit_default_options()
    opt.window = 3
    with pit.context_for(p, opt) as ctx:
        U = torch.empty(p.dof, dtype=torch.float64, device="cuda")
        pit.pit_fill_plain_guess(ctx, U)
        _, info_plain = pit.pit_solve(ctx, U)
    opt.window_start = pit.PIT_START_GIVEN
    rng = np.random.default_rng(52)
    for start, fewer in ((Uo + 1e-8 * rng.standard_normal(Uo.shape), True),
                         (1e3 * rng.standard_normal(Uo.shape), False)):
        with pit.context_for(p, opt) as ctx:
            U = _dev(start)
            status, info = pit.pit_solve(ctx, U)
            Ug = U.cpu().numpy().reshape(p.M, -1)
        assert info["converged"]
        assert np.abs(Ug - Uo).max() <= 1e-10 * np.abs(Uo).max()
        if fewer:
            assert info["newton_iters_total"] < info_plain["newton_iters_total"]
        else:
            assert info["windows"] > info["windows_converged"]  # the wild window was retried


def test_fma_probe_measures_a_plausible_rate():
    # GB300 runs FP64 at a small fraction of its FP32 rate; the probe must see both in range
    f64 = pit.pit_probe_fma_peak(0)
    f32 = pit.pit_probe_fma_peak(1)
    assert 0.3 < f64 < 3.0, f64
    assert 10.0 < f32 < 200.0 and f32 > 20 * f64, (f32, f64)


def test_wave_timers_report_every_team():
    # pit_wave_timers: 25 values per team of the last wavefront launch; the solved cells,
    # their sweeps and the cycle counters of the deep sweeps and of the level setup are
    # filled on the headline configuration (deep rows need teams of several CTAs)
    p = W.truncated(W.burgers256(0), 16)
    with pit.context_for(p) as ctx:
        U = torch.empty(p.dof, dtype=torch.float64, device="cuda")
        pit.pit_fill_plain_guess(ctx, U)
        status, info = pit.pit_solve(ctx, U)
        teams = pit.pit_wave_timers(ctx)
    assert len(teams) == info["wave_teams"] >= 1 and len(pit.WAVE_TIMER_NAMES) == 25
    assert all(t["total_ns"] > 0 for t in teams)
    # a team whose iterations find every level converged skips all its cells
    solved = [t for t in teams if t["cells"] > 0]
    assert solved
    for t in solved:
        assert t["sweeps"] >= t["cells"]
        assert t["setup_nodes_cyc"] > 0 and t["setup_teamreduce_cyc"] > 0 and t["sor_colour1_cyc"] > 0
