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
    solve_window: int = 0         # windows for the evaluation solves (0 = all levels at once)
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


def evaluate(cfg: LearnedConfig, net, probs):
    """Newton from the plain guess and from the learned guess for every problem."""
    import torch
    opt = pit.pit_default_options()
    opt.window = cfg.solve_window
    rows = []
    for p in probs:
        ctx = pit.context_for(p, opt)
        U = torch.empty((1, p.M, p.grid.ns), dtype=torch.float64, device="cuda")
        u0 = torch.as_tensor(np.ascontiguousarray(p.u0), device="cuda").reshape(1, -1)
        # plain guess
        pit.pit_fill_plain_guess(ctx, U.view(-1))
        st_p, info_p = pit.pit_solve(ctx, U.view(-1), check=False)
        U_plain = U.clone()
        # learned guess: network inference is part of the timed work
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        pit.pit_net_guess(net, u0, np.array([np.log10(p.params.mu_a)], dtype=np.float32), U)
        ev1.record()
        ev1.synchronize()
        ms_net = ev0.elapsed_time(ev1)
        st_l, info_l = pit.pit_solve(ctx, U.view(-1), check=False)
        diff = float((U - U_plain).abs().max() / U_plain.abs().max()) if st_p == 0 and st_l == 0 else float("nan")
        rows.append({"plain_ok": st_p == 0, "learned_ok": st_l == 0, "it_plain": info_p["newton_iters"],
                     "it_learned": info_l["newton_iters"], "ms_plain": info_p["ms_total"],
                     "ms_learned": info_l["ms_total"] + ms_net, "ms_net": ms_net, "diff": diff,
                     "res0_plain": info_p["res_inf"][0], "res0_learned": info_l["res_inf"][0]})
        ctx.close()
    return rows, U.view(p.M, -1).cpu().numpy()


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


def run(cfg: LearnedConfig) -> dict:
    import torch
    net = pit.pit_net_create(cfg.n, cfg.n, cfg.M, cfg.channels, cfg.blocks, max_batch=cfg.batch, seed=cfg.seed)
    train_probs = problems(cfg, 0, cfg.train)
    held = problems(cfg, 10_000_000, cfg.held_out)
    u0, lognu, targets, t_gen = generate(cfg, net, train_probs)
    losses, steps, t_train = train(cfg, net, u0, lognu, targets)
    rows, last_U = evaluate(cfg, net, held)
    del targets
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
        "max_rel_diff_solutions": max([r["diff"] for r in ok]) if ok else None,
        "check_problem": held[-1], "check_solution": last_U,
    }
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
