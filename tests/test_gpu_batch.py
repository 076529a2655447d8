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


@pytest.mark.parametrize("prec,team,window", [(0, 0, 0), (1, 0, 0), (0, 3, 2), (1, 5, 4)])
def test_batch_matches_oracle_per_problem(prec, team, window):
    probs = _problems()
    opt = pit.pit_default_options()
    opt.precision, opt.team_ctas, opt.window = prec, team, window
    with pit.pit_batch_create(probs, opt) as batch:
        results = []
        for rep in range(2):  # the second solve replays the captured graph
            status, info = pit.pit_batch_solve(batch)
            assert info["converged"] == len(probs)
            results.append([t["U"].cpu().numpy().copy() for t in batch.tensors])
        assert info["graph"] == 1
        for i, p in enumerate(probs):
            r = pit.pit_batch_result(batch, i)
            assert r["res_inf"] <= 1e-12
            Uo, _, _, _ = oracle.solve(p, tol=1e-13)
            Ug = results[-1][i].reshape(p.M, -1)
            assert np.abs(Ug - Uo).max() <= 1e-10 * np.abs(Uo).max(), (i, p.name)
            np.testing.assert_array_equal(results[0][i], results[1][i])
