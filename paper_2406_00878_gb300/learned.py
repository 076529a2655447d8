"""Learned initial guess for the all-at-once Newton solve.

A small residual conv net (``pit_net_*`` in libpit.so: BF16 tensor-core convs,
FP32 accumulation, Adam) is trained on space-time solutions that this solver
generates (``pit_batch_*``), then predicts the whole starting iterate of Newton
from (u^0, log10 nu). The converged solution does not depend on the start, so the
plain guess u^n = u^0 stays the fallback; the network only saves Newton work.

    python -m paper_2406_00878_gb300.learned [--n 128 --M 128 --train 4096 ...]

prints a JSON report: Newton iterations and converged DOF/s with the plain and
the learned starting iterate on held-out problems.
"""
from __future__ import annotations

import argparse
import json
import time
from dataclasses import dataclass, field

import numpy as np

from . import pit
from . import workloads as W


@dataclass
class LearnedConfig:
    n: int = 128                  # interior nodes per direction
    M: int = 128                  # time levels
    train: int = 4096             # training problems
    held_out: int = 256           # evaluation problems (other seeds)
    nu_range: tuple = (1e-3, 1e-1)
    dt: float = 1e-3
    channels: int = 64
    blocks: int = 4
    epochs: int = 8
    batch: int = 16
    lr: float = 1e-3
    seed: int = 0
    gen_window: int = 32          # windows for generating training solutions (robust Newton)
    solve_window: int = 0         # windows for the per-problem evaluation solves (0 = all levels at once)
    batch_window: int = 32        # windows of the batched evaluation forms
    batch_wave_nodes: int = 65536  # batched forms: grids of at least this many nodes are wavefront jobs
    chunk: int = 512              # problems per generation batch
    extra: dict = field(default_factory=dict)


def problems(cfg: LearnedConfig, first: int, count: int):
    """Burgers problems with a random sine-series u0 (modes k <= 8, a_k ~ N(0, 1/k^2))
    and nu log-uniform in nu_range; problem i uses seed cfg.seed * 1_000_003 + first + i."""
    out = []
    lo, hi = np.log10(cfg.nu_range[0]), np.log10(cfg.nu_range[1])
    for i in range(first, first + count):
        rng = np.random.default_rng(cfg.seed * 1_000_003 + i)
        g = W.Grid(cfg.n, cfg.n)
        nu = float(10.0 ** rng.uniform(lo, hi))
        out.append(W.Problem(f"learned{i}", g, W.Params(W.BURGERS, nu, 0.0), cfg.M, cfg.dt, W.fourier_u0(g, rng),
                             meta={"nu": nu, "index": i}))
    return out


def generate(cfg: LearnedConfig, net, probs):
    """Solve every problem with the batched solver; returns (u0 [S, Ns] FP64 CUDA,
    log10 nu [S] float32, targets BF16 CUDA [S, H, W, M], seconds)."""
    import torch
    S, Ns = len(probs), cfg.n * cfg.n
    u0 = torch.empty((S, Ns), dtype=torch.float64, device="cuda")
    targets = torch.empty((S, cfg.n, cfg.n, cfg.M), dtype=torch.bfloat16, device="cuda")
    lognu = np.array([np.log10(p.params.mu_a) for p in probs], dtype=np.float32)
    opt = pit.pit_default_options()
    opt.precision = pit.PIT_FP32_INNER
    opt.window = cfg.gen_window
    t0 = time.perf_counter()
    for c0 in range(0, S, cfg.chunk):
        part = probs[c0:c0 + cfg.chunk]
        with pit.pit_batch_create(part, opt) as batch:
            status, info = pit.pit_batch_solve(batch)
            for k, p in enumerate(part):
                t = batch.tensors[k]
                u0[c0 + k].copy_(t["u0"])
                pit.pit_net_make_target(net, t["u0"], t["U"], targets[c0 + k])
            torch.cuda.synchronize()
    return u0, lognu, targets, time.perf_counter() - t0


def train(cfg: LearnedConfig, net, u0, lognu, targets):
    import torch
    S = u0.shape[0]
    rng = np.random.default_rng(cfg.seed + 17)
    losses = []
    steps = 0
    t0 = time.perf_counter()
    for epoch in range(cfg.epochs):
        order = rng.permutation(S)
        for b0 in range(0, S - cfg.batch + 1, cfg.batch):
            idx = torch.as_tensor(order[b0:b0 + cfg.batch], device="cuda")
            # cosine decay of the learning rate over the run
            total = cfg.epochs * (S // cfg.batch)
            lr = cfg.lr * 0.5 * (1.0 + np.cos(np.pi * steps / max(total, 1)))
            want = (b0 == 0)
            loss = pit.pit_net_train_step(net, u0[idx].contiguous(), lognu[order[b0:b0 + cfg.batch]],
                                          targets[idx].contiguous(), max(lr, 1e-6), want_loss=want)
            if want:
                losses.append(loss)
            steps += 1
    torch.cuda.synchronize()
    return losses, steps, time.perf_counter() - t0


def infer(cfg: LearnedConfig, net, probs, out):
    """The network's starting iterates of all problems, cfg.batch at a time, into out
    [S, M * Ns] (FP64, CUDA). Returns the device time in ms."""
    import torch
    S, Ns = len(probs), cfg.n * cfg.n
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    u0 = torch.as_tensor(np.stack([np.ascontiguousarray(p.u0) for p in probs]), dtype=torch.float64, device="cuda")
    lognu = np.array([np.log10(p.params.mu_a) for p in probs], dtype=np.float32)
    ev0.record()
    for b0 in range(0, S, cfg.batch):
        B = min(cfg.batch, S - b0)
        pit.pit_net_guess(net, u0[b0:b0 + B], lognu[b0:b0 + B], out[b0:b0 + B].view(B, cfg.M, Ns))
    ev1.record()
    ev1.synchronize()
    return ev0.elapsed_time(ev1)


def _max_rel_diff(A, B, ok):
    """max over problems i with ok[i] of max|A_i - B_i| / max|B_i| (CUDA tensors [S, DOF])."""
    worst = 0.0
    for i in range(A.shape[0]):
        if ok[i]:
            worst = max(worst, float((A[i] - B[i]).abs().max() / B[i].abs().max()))
    return worst


def evaluate(cfg: LearnedConfig, net, probs):
    """Four forms of the solve on the same held-out problems, each to ||R||_inf <= 1e-12:

      plain     pit_solve per problem, FP64 level solves, plain guess u^n = u^0;
      learned   pit_solve per problem, FP64, from the network's guess (inference timed);
      learned_fp32  the same with FP32 level solves inside FP64 Newton;
      batched   one pit_batch launch for all problems, FP32 level solves inside FP64 Newton,
                windows of cfg.batch_window levels from the plain guess;
      combined  the network's guesses for all problems, then one pit_batch launch, FP32
                level solves, every window starting from the guess (PIT_START_GIVEN)
                (inference and the launch both timed).

    Returns (rows, forms, solutions): per-problem records of the per-problem forms, a
    summary per form, and the solutions of every form as CUDA tensors [S, M * Ns]."""
    import torch
    S, dof = len(probs), cfg.M * cfg.n * cfg.n
    sol = {k: torch.empty((S, dof), dtype=torch.float64, device="cuda")
           for k in ("plain", "learned", "learned_fp32", "batched", "combined")}
    guess = torch.empty((S, dof), dtype=torch.float64, device="cuda")
    infer(cfg, net, probs, guess)  # warm-up
    ms_net = infer(cfg, net, probs, guess)
    opt = pit.pit_default_options()
    opt.window = cfg.solve_window
    rows = []
    for i, p in enumerate(probs):
        ctx = pit.context_for(p, opt)
        U = sol["plain"][i]
        pit.pit_fill_plain_guess(ctx, U)
        st_p, info_p = pit.pit_solve(ctx, U, check=False)
        U = sol["learned"][i]
        U.copy_(guess[i])
        st_l, info_l = pit.pit_solve(ctx, U, check=False)
        rows.append({"plain_ok": st_p == 0, "learned_ok": st_l == 0, "it_plain": info_p["newton_iters"],
                     "it_learned": info_l["newton_iters"], "ms_plain": info_p["ms_total"],
                     "ms_learned": info_l["ms_total"] + ms_net / S, "ms_net": ms_net / S,
                     "res0_plain": info_p["res_inf"][0], "res0_learned": info_l["res_inf"][0]})
        ctx.close()
    # the learned guess with FP32 level solves, problem by problem (no batching)
    opt32 = pit.pit_default_options()
    opt32.window = cfg.solve_window
    opt32.precision = pit.PIT_FP32_INNER
    ms32, it32, ok32 = 0.0, [], 0
    for i, p in enumerate(probs):
        ctx = pit.context_for(p, opt32)
        U = sol["learned_fp32"][i]
        U.copy_(guess[i])
        st, info = pit.pit_solve(ctx, U, check=False)
        ms32 += info["ms_total"] + ms_net / S
        it32.append(info["newton_iters"])
        ok32 += st == 0
        ctx.close()
    ok = [r["plain_ok"] for r in rows]
    forms = {}
    n_ok = sum(ok)
    forms["plain"] = {"ms": sum(r["ms_plain"] for r in rows), "converged": n_ok,
                      "newton_iters_mean": float(np.mean([r["it_plain"] for r in rows]))}
    forms["learned"] = {"ms": sum(r["ms_learned"] for r in rows), "converged": sum(r["learned_ok"] for r in rows),
                        "newton_iters_mean": float(np.mean([r["it_learned"] for r in rows])), "ms_net": ms_net,
                        "max_rel_diff_vs_plain": _max_rel_diff(sol["learned"], sol["plain"], ok)}
    forms["learned_fp32"] = {"ms": ms32, "converged": ok32, "newton_iters_mean": float(np.mean(it32)),
                             "ms_net": ms_net, "max_rel_diff_vs_plain": _max_rel_diff(sol["learned_fp32"], sol["plain"], ok)}
    bopt = pit.pit_default_options()
    bopt.precision = pit.PIT_FP32_INNER
    bopt.window = cfg.batch_window
    bopt.batch_wave_nodes = cfg.batch_wave_nodes
    for name, start in (("batched", pit.PIT_START_PLAIN), ("combined", pit.PIT_START_GIVEN)):
        bopt.window_start = start
        Ub = sol[name]
        if start == pit.PIT_START_GIVEN:
            Ub.copy_(guess)
        with pit.pit_batch_create(probs, bopt, U=list(Ub)) as batch:
            # first solve: the launch is captured into a graph; time the replay after it
            ms_guess = infer(cfg, net, probs, Ub) if start == pit.PIT_START_GIVEN else 0.0
            pit.pit_batch_solve(batch, check=False)
            ms_guess = infer(cfg, net, probs, Ub) if start == pit.PIT_START_GIVEN else 0.0
            st, info = pit.pit_batch_solve(batch, check=False)
            its = [pit.pit_batch_result(batch, i)["newton_iters"] for i in range(S)]
        forms[name] = {"ms": info["ms"] + ms_guess, "ms_launch": info["ms"], "ms_net": ms_guess,
                       "converged": info["converged"], "graph_replay": bool(info["graph"]),
                       "newton_iters_mean": float(np.mean(its)), "window": cfg.batch_window,
                       "max_rel_diff_vs_plain": _max_rel_diff(Ub, sol["plain"], ok)}
    for f in forms.values():
        f["dof_per_s"] = dof * S / (f["ms"] * 1e-3) if f["ms"] > 0 else None
    return rows, forms, sol


def train_flops_per_step(cfg: LearnedConfig) -> float:
    """Tensor-core flops (FMA = 2) of one training step: forward, data gradients of all
    layers but the input one, weight gradients of all layers (input channels padded to 16)."""
    pix = cfg.batch * cfg.n * cfg.n
    C, M = cfg.channels, cfg.M
    fwd = [(16, C)] + [(C, C)] * (2 * cfg.blocks) + [(C, M)]
    per = lambda ci, co: 2.0 * pix * co * 9 * ci
    f = sum(per(ci, co) for ci, co in fwd)          # forward
    f += sum(per(ci, co) for ci, co in fwd[1:])     # data gradients
    f += sum(per(ci, co) for ci, co in fwd)         # weight gradients
    return f


def run(cfg: LearnedConfig, keep_solutions: bool = False) -> dict:
    import torch
    net = pit.pit_net_create(cfg.n, cfg.n, cfg.M, cfg.channels, cfg.blocks, max_batch=cfg.batch, seed=cfg.seed)
    train_probs = problems(cfg, 0, cfg.train)
    held = problems(cfg, 10_000_000, cfg.held_out)
    u0, lognu, targets, t_gen = generate(cfg, net, train_probs)
    losses, steps, t_train = train(cfg, net, u0, lognu, targets)
    del targets, u0
    rows, forms, sol = evaluate(cfg, net, held)
    net.close()
    torch.cuda.synchronize()
    ok = [r for r in rows if r["plain_ok"] and r["learned_ok"]]
    dof = cfg.n * cfg.n * cfg.M
    flops_step = train_flops_per_step(cfg)
    rep = {
        "config": {k: v for k, v in cfg.__dict__.items() if k != "extra"},
        "generation_s": t_gen, "generation_dof_per_s": cfg.train * dof / t_gen, "training_s": t_train,
        "train_steps": steps, "train_tflops": flops_step * steps / t_train / 1e12,
        "loss_first": losses[0] if losses else None, "loss_last": losses[-1] if losses else None,
        "held_out_converged_plain": sum(r["plain_ok"] for r in rows),
        "held_out_converged_learned": sum(r["learned_ok"] for r in rows),
        "newton_iters_plain_mean": float(np.mean([r["it_plain"] for r in ok])) if ok else None,
        "newton_iters_learned_mean": float(np.mean([r["it_learned"] for r in ok])) if ok else None,
        "residual0_plain_mean": float(np.mean([r["res0_plain"] for r in ok])) if ok else None,
        "residual0_learned_mean": float(np.mean([r["res0_learned"] for r in ok])) if ok else None,
        "dof_per_s_plain": dof * len(ok) / (sum(r["ms_plain"] for r in ok) * 1e-3) if ok else None,
        "dof_per_s_learned": dof * len(ok) / (sum(r["ms_learned"] for r in ok) * 1e-3) if ok else None,
        "ms_net_mean": float(np.mean([r["ms_net"] for r in rows])),
        "max_rel_diff_solutions": forms["learned"]["max_rel_diff_vs_plain"],
        "forms": forms,
        "check_problem": held[-1], "check_solution": sol["learned"][-1].view(cfg.M, -1).cpu().numpy(),
    }
    if keep_solutions:
        rep["held_out"] = held
        rep["solutions"] = sol
    return rep


def main():
    ap = argparse.ArgumentParser()
    for f, v in LearnedConfig().__dict__.items():
        if isinstance(v, (int, float)) and not isinstance(v, bool):
            ap.add_argument("--" + f.replace("_", "-"), type=type(v), default=v)
    args = ap.parse_args()
    cfg = LearnedConfig(**{k: getattr(args, k) for k in LearnedConfig().__dict__ if hasattr(args, k)})
    rep = run(cfg)
    rep.pop("check_problem")
    rep.pop("check_solution")
    print(json.dumps(rep))


if __name__ == "__main__":
    main()
