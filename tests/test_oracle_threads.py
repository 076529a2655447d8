"""The oracle's timing build (OpenMP over element-independent loops) must return the
same bits as the tested single-threaded build: it only decides which host thread
computes which level, row or vector entry, never the order of a sum."""
import numpy as np
import pytest

import oracle
from paper_2406_00878_gb300 import workloads as W


@pytest.fixture
def threads():
    n = oracle.use_threads(4)
    yield n
    oracle.use_threads(1)


def _run(p):
    R = oracle.residual(p.grid, p.params, p.M, p.dt, p.u0, p.plain_guess() * 0.9, p.bc, p.q)
    C = oracle.jacobian(p.grid, p.params, p.M, p.dt, p.plain_guess() * 1.1, p.bc)
    U, it, res, upd = oracle.solve(p, tol=1e-12)
    return R, C, U, it, res


@pytest.mark.parametrize("make", [
    # 130 x 131 nodes (> 16384): the BiCGStab level solves take their threaded branches
    lambda: W.random_problem(31, 130, 131, 3, W.BURGERS, with_bc=True, with_q=True),
    lambda: W.heat32(0),
])
def test_threaded_oracle_is_bitwise_the_single_threaded_one(make, threads):
    p = make()
    oracle.use_threads(1)
    ref = _run(p)
    assert oracle.use_threads(4) >= 1
    got = _run(p)
    for a, b in zip(ref, got):
        assert np.array_equal(np.asarray(a), np.asarray(b))
