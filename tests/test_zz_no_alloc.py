"""pit_block_solve_noalloc -- the block solve for callers that cannot allocate device
memory -- must give the context-based pit_block_solve's result on the same inputs,
call after call, while its workspace is the library's static device array.

Runs last (file name) so that a failure here stops a `-x` run only after every
other test has run; it also passes alone in a fresh process."""
import numpy as np
import pytest

from paper_2406_00878_gb300 import pit
from paper_2406_00878_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("seed,nx,ny,M,eq", [(21, 40, 33, 4, W.BURGERS), (22, 29, 36, 3, W.HEAT),
                                             (23, 256, 256, 3, W.BURGERS)])
def test_noalloc_block_solve_matches_block_solve_twice(seed, nx, ny, M, eq):
    p = W.random_problem(seed, nx, ny, M, eq, with_bc=True)
    rng = np.random.default_rng(seed)
    U = _dev(p.plain_guess() + 0.05 * rng.standard_normal((M, p.grid.ns)))
    R = _dev(rng.standard_normal((M, p.grid.ns)))
    with pit.context_for(p) as ctx:
        coef = torch.empty(5 * p.dof, dtype=torch.float64, device="cuda")
        pit.pit_assemble(ctx, U, coef)
        ref = torch.empty(p.dof, dtype=torch.float64, device="cuda")
        pit.pit_block_solve(ctx, U, R, ref, eta=1e-14)
    ref = ref.cpu().numpy()
    tol = 1e-10 * np.abs(ref).max()
    for _ in range(2):
        dU = torch.full((p.dof,), float("nan"), dtype=torch.float64, device="cuda")
        status, msg = pit.pit_block_solve_noalloc(nx, ny, M, coef, R, dU, eta=1e-14)
        assert status == pit.PIT_OK, msg
        np.testing.assert_allclose(dU.cpu().numpy(), ref, rtol=0, atol=tol)


def test_noalloc_rejects_sizes_beyond_its_workspace():
    t = torch.zeros(5, dtype=torch.float64, device="cuda")
    s, msg = pit.pit_block_solve_noalloc(pit.PIT_NOALLOC_MAX_NX + 1 if hasattr(pit, "PIT_NOALLOC_MAX_NX") else 513,
                                         1, 1, t.repeat(513), t[:1].repeat(513), t[:1].repeat(513), check=False)
    assert s == pit.PIT_EUNSUPPORTED and "PIT_NOALLOC_MAX_NX" in msg
    s, msg = pit.pit_block_solve_noalloc(1, 1, 4097, t.repeat(4097), t[:1].repeat(4097), t[:1].repeat(4097),
                                         check=False)
    assert s == pit.PIT_EUNSUPPORTED and "PIT_NOALLOC_MAX_LEVELS" in msg


def test_noalloc_reports_a_nan_coefficient_as_diverged():
    # a NaN entry must reach the caller as PIT_EDIVERGED, both with the automatic
    # solver choice (the level's bound is then NaN) and with SOR forced
    p = W.random_problem(24, 31, 27, 3, W.BURGERS)
    U = _dev(p.plain_guess())
    R = _dev(np.random.default_rng(24).standard_normal((3, p.grid.ns)))
    with pit.context_for(p) as ctx:
        coef = torch.empty(5 * p.dof, dtype=torch.float64, device="cuda")
        pit.pit_assemble(ctx, U, coef)
    coef[3 * p.dof + p.grid.ns + 17] = float("nan")  # an S entry of level 2
    for solver in (pit.PIT_LIN_AUTO, pit.PIT_LIN_SOR):
        opt = pit.pit_default_options()
        opt.lin_solver = solver
        dU = torch.zeros(p.dof, dtype=torch.float64, device="cuda")
        status, msg = pit.pit_block_solve_noalloc(31, 27, 3, coef, R, dU, eta=1e-14, opt=opt, check=False)
        assert status == pit.PIT_EDIVERGED, (solver, status, msg)


def test_noalloc_refuses_a_capturing_stream():
    # every call reads its status back and synchronises, which a graph capture forbids
    p = W.random_problem(25, 16, 16, 2, W.HEAT)
    t = torch.zeros(5 * p.dof, dtype=torch.float64, device="cuda")
    R = torch.zeros(p.dof, dtype=torch.float64, device="cuda")
    dU = torch.zeros(p.dof, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    out = {}
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            out["r"] = pit.pit_block_solve_noalloc(16, 16, 2, t, R, dU, eta=1e-14, stream=s, check=False)
        finally:
            g.capture_end()
    status, msg = out["r"]
    assert status == pit.PIT_EUNSUPPORTED and "captured" in msg
