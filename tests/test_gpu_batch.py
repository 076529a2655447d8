"""f2: many independent problems in one persistent launch (teams of CTAs placed by
the autotuner's schedule), replayed from a CUDA graph; every problem must match the
FP64 oracle to 1e-10 relative."""
import numpy as np
import pytest

import oracle
from paper_2406_00878_gb300 import pit
from paper_2406_00878_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problems():
    return [
        W.random_problem(61, 24, 30, 5, W.BURGERS, with_bc=True, with_q=True),
        W.random_problem(62, 40, 17, 7, W.HEAT, with_bc=True),
        W.random_problem(63, 9, 13, 3, W.BURGERS),
        W.heat32(4),
        W.random_problem(64, 33, 33, 9, W.HEAT, with_q=True, mu_b=0.0),
        W.truncated(W.burgers256(0), 3),
    ]


def _wave_job(p, wave_nodes):
    return wave_nodes > 0 and p.grid.nx * p.grid.ny >= wave_nodes


# wave = batch_wave_nodes: 65536 (default) makes the 256 x 256 problem a wavefront job
# (several teams, Newton iterations in flight) and packs the rest; 0 packs every
# problem; 1 makes every problem a wavefront job
@pytest.mark.parametrize("prec,team,window,wave", [(0, 0, 0, 65536), (1, 0, 0, 0), (0, 3, 2, 0), (1, 5, 4, 65536),
                                                   (1, 0, 4, 1), (0, 0, 2, 1)])
def test_batch_matches_oracle_per_problem(prec, team, window, wave):
    probs = _problems()
    opt = pit.pit_default_options()
    assert opt.batch_wave_nodes == 65536
    opt.precision, opt.team_ctas, opt.window, opt.batch_wave_nodes = prec, team, window, wave
    with pit.pit_batch_create(probs, opt) as batch:
        for i, p in enumerate(probs):
            where = pit.pit_batch_placement(batch, i)
            assert (where["teams"] > 1) == _wave_job(p, wave), (i, where)
            assert where["team_ctas"] >= 1 and where["teams"] * where["team_ctas"] <= 160
        results = []
        for rep in range(2):  # the second solve replays the captured graph
            status, info = pit.pit_batch_solve(batch)
            assert info["converged"] == len(probs)
            results.append([t["U"].cpu().numpy().copy() for t in batch.tensors])
        assert info["graph"] == 1
        assert info["wave_jobs"] == sum(_wave_job(p, wave) for p in probs)
        for i, p in enumerate(probs):
            r = pit.pit_batch_result(batch, i)
            assert r["res_inf"] <= 1e-12
            Uo, _, _, _ = oracle.solve(p, tol=1e-13)
            Ug = results[-1][i].reshape(p.M, -1)
            assert np.abs(Ug - Uo).max() <= 1e-10 * np.abs(Uo).max(), (i, p.name)
            np.testing.assert_array_equal(results[0][i], results[1][i])


@pytest.mark.parametrize("wave", [0, 1])
def test_batch_unconverged_problems_report_their_true_residual(wave):
    """With two Newton updates allowed, no problem converges: the batch says so, and the
    residual it reports for each is the oracle's residual of the U it returned."""
    probs = _problems()[:4]
    opt = pit.pit_default_options()
    opt.newton_max, opt.batch_wave_nodes, opt.window = 2, wave, 4
    with pit.pit_batch_create(probs, opt) as batch:
        status, info = pit.pit_batch_solve(batch, check=False)
        assert status == pit.PIT_ENOCONV and info["converged"] < len(probs)
        assert info["wave_jobs"] == (len(probs) if wave else 0)
        for i, p in enumerate(probs):
            r = pit.pit_batch_result(batch, i)
            U = batch.tensors[i]["U"].cpu().numpy().reshape(p.M, -1)
            R = oracle.residual(p.grid, p.params, p.M, p.dt, p.u0, U, p.bc, p.q)
            ro = float(np.abs(R).max())
            assert abs(r["res_inf"] - ro) <= 1e-9 * ro + 1e-15, (i, r["res_inf"], ro)


def _source_driven_burgers():
    """Burgers on 32 x 32, nu = 0.02, tau = 0.05, u0 = 0, a steady source
    50 sin(2 pi x) sin(pi y): u grows to ~6 over 8 levels (cell Reynolds/CFL ~10).
    The oracle's all-at-once Newton from the plain guess converges on windows of 1, 2
    and 4 levels (6, 7, 9 updates) but diverges on all 8 (residual past 1e12)."""
    g = W.Grid(32, 32)
    X, Y = g.nodes()
    q = np.tile((50.0 * np.sin(2 * np.pi * X) * np.sin(np.pi * Y)).ravel(), (8, 1))
    return W.Problem("burgers_source32x8", g, W.Params(W.BURGERS, 0.02, 0.0), 8, 0.05, np.zeros(g.ns), None,
                     np.ascontiguousarray(q))


@pytest.mark.parametrize("wave", [0, 1])
def test_batch_restarts_diverged_windows(wave):
    """A window whose Newton diverges is restarted shorter, in a packed team and in a
    wavefront job (whose teams all leave the window and restart their synchronisation).
    A problem with a NaN in u0 diverges in every window and ends unconverged without
    disturbing the others."""
    div = _source_driven_burgers()
    for Mw, ok_ in ((4, True), (8, False)):
        _, it, res, _ = oracle.newton_all_at_once(div.grid, div.params, Mw, div.dt, div.u0, np.tile(div.u0, Mw),
                                                  q=div.q[:Mw], maxit=30)
        assert (it >= 0) == ok_ and (ok_ or not (np.nanmax(res) < 1e10))
    nan = W.truncated(W.burgers256(0), 3)
    nan.u0 = nan.u0.copy()
    nan.u0[1000] = np.nan
    ok = W.random_problem(63, 9, 13, 3, W.BURGERS)
    probs = [div, nan, ok]
    opt = pit.pit_default_options()
    opt.window, opt.batch_wave_nodes = 8, wave
    with pit.pit_batch_create(probs, opt) as batch:
        for rep in range(2):
            status, info = pit.pit_batch_solve(batch, check=False)
            r = [pit.pit_batch_result(batch, i) for i in range(3)]
            assert status == pit.PIT_ENOCONV and info["converged"] == 2, (status, r)
            assert info["wave_jobs"] == (3 if wave else 0)
            assert not (r[1]["res_inf"] <= 1e-12)
            for i in (0, 2):
                p = probs[i]
                assert r[i]["res_inf"] <= 1e-12
                Uo = oracle.sequential_bdf1(p.grid, p.params, p.M, p.dt, p.u0, p.bc, p.q)[0]
                Ug = batch.tensors[i]["U"].cpu().numpy().reshape(p.M, -1)
                assert np.abs(Ug - Uo).max() <= 1e-10 * np.abs(Uo).max(), (i, rep)
            # the first window (all 8 levels) did not converge: it was split
            assert r[0]["windows_converged"] > 1, r[0]


@pytest.mark.parametrize("wave", [0, 1])
def test_batch_wait_timeout_is_reported_and_the_device_stays_usable(wave):
    """A wait budget of one poll: the first team or job wait that is not satisfied at
    once gives up, the launch ends with PIT_ETIMEOUT (no fault, no hang), and a fresh
    batch on the same device then solves to the oracle's solution."""
    probs = _problems()[:3]
    opt = pit.pit_default_options()
    opt.wait_budget, opt.team_ctas, opt.batch_wave_nodes = 1, 4, wave  # fixed teams: no autotuner runs
    with pit.pit_batch_create(probs, opt) as batch:
        status, _ = pit.pit_batch_solve(batch, check=False)
        assert status == pit.PIT_ETIMEOUT, status
        assert "budget" in pit.lib().pit_batch_last_error(batch.handle).decode()
    opt = pit.pit_default_options()
    opt.batch_wave_nodes = wave
    with pit.pit_batch_create(probs[:1], opt) as batch:
        status, info = pit.pit_batch_solve(batch)
        assert info["converged"] == 1
        Uo, _, _, _ = oracle.solve(probs[0], tol=1e-13)
        Ug = batch.tensors[0]["U"].cpu().numpy().reshape(probs[0].M, -1)
        assert np.abs(Ug - Uo).max() <= 1e-10 * np.abs(Uo).max()


def _closure_problem(bit, seed):
    """A small problem of one closure: bit = closure index 2 conv + nlv."""
    conv, nlv = bool(bit & 2), bool(bit & 1)
    eq = W.BURGERS if conv else W.HEAT
    return W.random_problem(seed, 11, 9, 3, eq, with_bc=bool(seed & 1), mu_a=0.05 if conv else 0.5,
                            mu_b=(0.3 if nlv else 0.0))


@pytest.mark.parametrize("prec", [0, 1])
def test_every_closure_set_is_solved(prec):
    """Each of the 15 non-empty sets of closures (Burgers/heat x constant/variable
    viscosity), per precision: one problem of every closure in the set, each equal to the
    oracle's solution. A batch of several closures runs one launch per closure, each with
    the kernel compiled for that closure alone."""
    for closures in range(1, 16):
        probs = [_closure_problem(c, 100 + 4 * closures + c) for c in range(4) if closures >> c & 1]
        opt = pit.pit_default_options()
        opt.precision, opt.team_ctas, opt.batch_wave_nodes = prec, 2, 0
        with pit.pit_batch_create(probs, opt) as batch:
            status, info = pit.pit_batch_solve(batch)
            assert info["converged"] == len(probs), closures
            for i, p in enumerate(probs):
                Uo, _, _, _ = oracle.solve(p, tol=1e-13)
                Ug = batch.tensors[i]["U"].cpu().numpy().reshape(p.M, -1)
                assert np.abs(Ug - Uo).max() <= 1e-10 * np.abs(Uo).max(), (closures, i)


def test_full_size_batched_workload_every_problem_against_the_oracle():
    # the 64-problem batched workload at full size, in the configuration the benchmark
    # times (FP32 level solves, windows of 32, grids of 256^2 and up as wavefront jobs):
    # for EVERY problem the oracle's residual of the returned solution at every level,
    # and its first two levels against the oracle's own solve of those levels
    import os
    probs = W.batched(0)
    opt = pit.pit_default_options()
    opt.precision = pit.PIT_FP32_INNER
    opt.window = 32
    with pit.pit_batch_create(probs, opt) as batch:
        status, info = pit.pit_batch_solve(batch)
        assert info["converged"] == len(probs)
        sols = [t["U"].cpu().numpy().reshape(p.M, -1) for t, p in zip(batch.tensors, probs)]
    oracle.use_threads(len(os.sched_getaffinity(0)))   # bitwise the single-threaded oracle
    try:
        for i, (p, Ug) in enumerate(zip(probs, sols)):
            R = oracle.residual(p.grid, p.params, p.M, p.dt, p.u0, Ug, p.bc, p.q)
            assert np.isfinite(R).all() and np.abs(R).max() <= 2e-12, (i, float(np.abs(R).max()))
            Uo, _, _, _ = oracle.solve(W.truncated(p, 2), tol=1e-13)
            assert np.abs(Ug[:2] - Uo).max() <= 1e-10 * np.abs(Uo).max(), (i, p.name)
    finally:
        oracle.use_threads(1)


@pytest.mark.parametrize("wave", [0, 1])
def test_batch_starts_windows_from_the_given_iterate(wave):
    # window_start = PIT_START_GIVEN: each window starts from the iterate the caller left in
    # U. From a slightly perturbed solution Newton needs fewer updates than from the plain
    # guess and reaches the same solution; from a wild start on one problem the window
    # diverges, is retried from the plain guess, and still reaches the oracle's solution.
    probs = _problems()[:4]
    opt = pit.pit_default_options()
    opt.window, opt.batch_wave_nodes = 3, wave
    with pit.pit_batch_create(probs, opt) as batch:
        pit.pit_batch_solve(batch)
        exact = [t["U"].clone() for t in batch.tensors]
        plain_iters = [pit.pit_batch_result(batch, i)["newton_iters"] for i in range(len(probs))]
    opt.window_start = pit.PIT_START_GIVEN
    gen = torch.Generator(device="cuda").manual_seed(7)
    starts = [u + 1e-7 * u.abs().max() * torch.randn(u.shape, generator=gen, device="cuda", dtype=torch.float64)
              for u in exact]
    starts[2] = 1e3 * torch.randn(exact[2].shape, generator=gen, device="cuda", dtype=torch.float64)
    Us = [s.clone() for s in starts]
    with pit.pit_batch_create(probs, opt, U=Us) as batch:
        # the autotuner's calibration runs must leave the given iterates alone
        for u, s in zip(Us, starts):
            assert torch.equal(u, s)
        status, info = pit.pit_batch_solve(batch)
        assert info["converged"] == len(probs)
        given_iters = [pit.pit_batch_result(batch, i)["newton_iters"] for i in range(len(probs))]
        for i, p in enumerate(probs):
            Uo, _, _, _ = oracle.solve(p, tol=1e-13)
            Ug = Us[i].cpu().numpy().reshape(p.M, -1)
            assert np.abs(Ug - Uo).max() <= 1e-10 * np.abs(Uo).max(), (i, p.name)
    for i in (0, 1, 3):
        assert given_iters[i] < plain_iters[i], (i, given_iters, plain_iters)
