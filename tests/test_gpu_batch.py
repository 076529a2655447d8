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


# solo = batch_solo_nodes: 65536 (default) sends the 256 x 256 problem through the
# wavefront path and packs the rest; 0 packs every problem; 1 solves every one alone
@pytest.mark.parametrize("prec,team,window,solo", [(0, 0, 0, 65536), (1, 0, 0, 0), (0, 3, 2, 0), (1, 5, 4, 65536),
                                                   (1, 0, 4, 1), (0, 0, 2, 1)])
def test_batch_matches_oracle_per_problem(prec, team, window, solo):
    probs = _problems()
    opt = pit.pit_default_options()
    assert opt.batch_solo_nodes == 65536
    opt.precision, opt.team_ctas, opt.window, opt.batch_solo_nodes = prec, team, window, solo
    with pit.pit_batch_create(probs, opt) as batch:
        for i, p in enumerate(probs):
            where = pit.pit_batch_placement(batch, i)
            assert where["solo"] == (solo > 0 and p.grid.nx * p.grid.ny >= solo), (i, where)
            assert where["team_ctas"] >= 1 and where["teams"] >= 1
        results = []
        for rep in range(2):  # the second solve replays the captured graph
            status, info = pit.pit_batch_solve(batch)
            assert info["converged"] == len(probs)
            results.append([t["U"].cpu().numpy().copy() for t in batch.tensors])
        n_solo = sum(solo > 0 and p.grid.nx * p.grid.ny >= solo for p in probs)
        assert info["solo"] == n_solo
        assert info["graph"] == (1 if n_solo < len(probs) else 0)
        assert info["ms"] >= info["ms_solo"] + info["ms_packed"] - 1e-3
        for i, p in enumerate(probs):
            r = pit.pit_batch_result(batch, i)
            assert r["res_inf"] <= 1e-12
            Uo, _, _, _ = oracle.solve(p, tol=1e-13)
            Ug = results[-1][i].reshape(p.M, -1)
            assert np.abs(Ug - Uo).max() <= 1e-10 * np.abs(Uo).max(), (i, p.name)
            np.testing.assert_array_equal(results[0][i], results[1][i])


@pytest.mark.parametrize("solo", [0, 1])
def test_batch_unconverged_problems_report_their_true_residual(solo):
    """With one Newton update allowed, no problem converges: the batch says so, and the
    residual it reports for each is the oracle's residual of the U it returned (for a
    solo problem that stopped early, taken over all levels)."""
    probs = _problems()[:4]
    opt = pit.pit_default_options()
    opt.newton_max, opt.batch_solo_nodes, opt.window = 1, solo, 4
    with pit.pit_batch_create(probs, opt) as batch:
        status, info = pit.pit_batch_solve(batch, check=False)
        assert status == pit.PIT_ENOCONV and info["converged"] < len(probs)
        for i, p in enumerate(probs):
            r = pit.pit_batch_result(batch, i)
            U = batch.tensors[i]["U"].cpu().numpy().reshape(p.M, -1)
            R = oracle.residual(p.grid, p.params, p.M, p.dt, p.u0, U, p.bc, p.q)
            ro = float(np.abs(R).max())
            assert abs(r["res_inf"] - ro) <= 1e-9 * ro + 1e-15, (i, r["res_inf"], ro)
