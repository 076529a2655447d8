"""Child process of test_gpu_bounds_check.py: loads the bounds-checking build of the
library (given on the command line) and runs every kernel family on tiny and ragged
shapes against the FP64 oracle, reading the bounds record after each call. Prints one
JSON line per check: {"name", "err", "tol", "bounds": [enabled, first_id]}.

Not a test module itself (its name does not start with test_): it must run in a fresh
process, since a process holds one library."""
import json
import sys

import numpy as np
import torch

import oracle
from paper_2406_00878_gb300 import pit
from paper_2406_00878_gb300 import workloads as W


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def _emit(name, err, tol):
    en, fid = pit.pit_bounds_status()
    print(json.dumps({"name": name, "err": float(err), "tol": float(tol), "bounds": [en, fid]}), flush=True)


# (seed, nx, ny, M, equation, bc, q): one node, a ragged tiny grid, a single column, a
# single row, and grids that split into several row strips (team sizes below)
SHAPES = [
    (1, 1, 1, 1, W.HEAT, False, False),
    (2, 3, 5, 2, W.BURGERS, True, True),
    (6, 1, 37, 3, W.HEAT, True, True),
    (7, 41, 1, 3, W.BURGERS, True, False),
    (3, 17, 33, 3, W.HEAT, True, False),
    (9, 40, 48, 4, W.BURGERS, True, True),
]


def _problem(c):
    seed, nx, ny, M, eq, bc, q = c
    return W.random_problem(seed, nx, ny, M, eq, with_bc=bc, with_q=q)


def _stages(c):
    p = _problem(c)
    tag = f"{p.grid.nx}x{p.grid.ny}x{p.M}"
    rng = np.random.default_rng(c[0] + 100)
    U = np.ascontiguousarray(p.plain_guess() + 0.05 * rng.standard_normal((p.M, p.grid.ns)))
    R = rng.standard_normal((p.M, p.grid.ns))
    with pit.context_for(p) as ctx:
        Rg = torch.empty(p.dof, dtype=torch.float64, device="cuda")
        pit.pit_residual(ctx, _dev(U), Rg)
        Ro = oracle.residual(p.grid, p.params, p.M, p.dt, p.u0, U, p.bc, p.q)
        _emit(f"residual {tag}", np.abs(Rg.cpu().numpy().reshape(p.M, -1) - Ro).max(), 1e-12 * max(np.abs(Ro).max(), 1))
        coef = torch.empty(5 * p.dof, dtype=torch.float64, device="cuda")
        pit.pit_assemble(ctx, _dev(U), coef)
        co = np.asarray(oracle.jacobian(p.grid, p.params, p.M, p.dt, U, p.bc))
        _emit(f"assemble {tag}", np.abs(coef.cpu().numpy().reshape(5, p.M, -1) - co).max(),
              1e-13 * max(np.abs(co).max(), 1.0))
    do = oracle.block_solve(p.grid.nx, p.grid.ny, p.M, oracle.jacobian(p.grid, p.params, p.M, p.dt, U, p.bc), R,
                            solver=oracle.SOLVER_BAND_LU)
    for team in (0, 1, 3, 8):
        if team > p.grid.ny:
            continue
        for solver in (pit.PIT_LIN_SOR, pit.PIT_LIN_BICGSTAB):
            opt = pit.pit_default_options()
            opt.team_ctas, opt.lin_solver, opt.lin_max_iter = team, solver, 20000
            with pit.context_for(p, opt) as ctx:
                dU = torch.empty(p.dof, dtype=torch.float64, device="cuda")
                pit.pit_block_solve(ctx, _dev(U), _dev(R), dU, eta=1e-14)
                err = np.abs(dU.cpu().numpy().reshape(p.M, -1) - do).max()
            _emit(f"block_solve {tag} team={team} solver={solver}", err, 1e-10 * max(np.abs(do).max(), 1e-300))
    # the context-free block solve on the same system
    coef_o = np.asarray(oracle.jacobian(p.grid, p.params, p.M, p.dt, U, p.bc))
    dU = torch.full((p.dof,), float("nan"), dtype=torch.float64, device="cuda")
    status, msg = pit.pit_block_solve_noalloc(p.grid.nx, p.grid.ny, p.M, _dev(coef_o), _dev(R), dU, eta=1e-14)
    err = np.abs(dU.cpu().numpy().reshape(p.M, -1) - do).max() if status == pit.PIT_OK else float("inf")
    _emit(f"noalloc {tag}", err, 1e-10 * max(np.abs(do).max(), 1e-300))


def _solves(c):
    p = _problem(c)
    tag = f"{p.grid.nx}x{p.grid.ny}x{p.M}"
    Uo, _, _, _ = oracle.solve(p, tol=1e-13)
    tol = 1e-10 * max(np.abs(Uo).max(), 1e-300)
    # (wave_teams, team_ctas, precision, window): the per-stage path (-1), wavefront launches
    # with one and several teams (deep rows on the wider strips), FP32 level solves, windows
    for teams, team, prec, window in [(-1, 0, 0, 0), (1, 0, 0, 0), (3, 0, 0, 0), (2, 8, 0, 0), (2, 0, 1, 0),
                                      (3, 8, 1, 0), (2, 0, 0, 2)]:
        if team > p.grid.ny:
            continue
        opt = pit.pit_default_options()
        opt.wave_teams, opt.team_ctas, opt.precision, opt.window = teams, team, prec, window
        with pit.context_for(p, opt) as ctx:
            U = torch.empty(p.dof, dtype=torch.float64, device="cuda")
            pit.pit_fill_plain_guess(ctx, U)
            status, info = pit.pit_solve(ctx, U, check=False)
            err = np.abs(U.cpu().numpy().reshape(p.M, -1) - Uo).max() if status == pit.PIT_OK else float("inf")
        _emit(f"solve {tag} teams={teams} team={team} prec={prec} window={window}", err, tol)


def _batches():
    probs = [_problem(c) for c in SHAPES]
    refs = [oracle.solve(p, tol=1e-13)[0] for p in probs]
    for prec, wave, window in [(0, 0, 0), (1, 0, 2), (0, 1, 0), (1, 1, 0)]:
        opt = pit.pit_default_options()
        opt.precision, opt.batch_wave_nodes, opt.window = prec, wave, window
        with pit.pit_batch_create(probs, opt) as batch:
            status, info = pit.pit_batch_solve(batch, check=False)
            for i, (p, Uo) in enumerate(zip(probs, refs)):
                Ug = batch.tensors[i]["U"].cpu().numpy().reshape(p.M, -1)
                err = np.abs(Ug - Uo).max() if status == pit.PIT_OK else float("inf")
                _emit(f"batch prec={prec} wave={wave} window={window} problem={i}", err,
                      1e-10 * max(np.abs(Uo).max(), 1e-300))


def main():
    pit.use_library(sys.argv[1])
    en, fid = pit.pit_bounds_status()
    print(json.dumps({"name": "loaded", "err": 0.0, "tol": 0.0, "bounds": [en, fid]}), flush=True)
    for c in SHAPES:
        _stages(c)
        _solves(c)
    _batches()


if __name__ == "__main__":
    main()
