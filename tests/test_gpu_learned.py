"""f3: the learned initial guess. The BF16 tensor-core network against the FP64
oracle (forward values and every layer's gradient), Adam training, and the gain of
the trained network as Newton's starting iterate over the plain guess.

BF16 tolerances: activations and weights carry 8 significant bits, so a layer's
output differs from FP64 by ~0.4 % per rounding; through the network the relative
error in norm stays below 3 % (forward) and gradients keep a cosine similarity
above 0.995 with the oracle's."""
import numpy as np
import pytest

import oracle
from oracle import convnet as CN
from paper_2406_00878_gb300 import learned
from paper_2406_00878_gb300 import pit
from paper_2406_00878_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _bf16_round(a):
    return torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _setup(seed=0, H=6, Wd=10, M=16, C=16, blocks=2, B=3):
    rng = np.random.default_rng(seed)
    shapes = CN.layer_shapes(C, blocks, M)
    theta = np.concatenate([np.concatenate([0.3 * rng.standard_normal(co * 9 * ci), 0.05 * rng.standard_normal(co)])
                            for co, ci in shapes]).astype(np.float32)
    u0 = rng.standard_normal((B, H * Wd))
    lognu = rng.uniform(-3, -1, B).astype(np.float32)
    target = rng.standard_normal((B, H, Wd, M)) * 0.5
    net = pit.pit_net_create(H, Wd, M, C, blocks, max_batch=B, seed=1)
    pit.pit_net_set_params(net, theta)
    return net, shapes, theta, u0, lognu, target


def test_forward_matches_oracle():
    net, shapes, theta, u0, lognu, target = _setup()
    B, Ns = u0.shape
    H, Wd, M = net.shape.height, net.shape.width, net.shape.levels
    with net:
        U = torch.empty((B, M, Ns), dtype=torch.float64, device="cuda")
        u0_d = torch.as_tensor(u0, device="cuda")
        pit.pit_net_guess(net, u0_d, lognu, U)
        corr = (U.cpu().numpy() - u0[:, None, :]).reshape(B, M, H, Wd).transpose(0, 2, 3, 1)
    params = CN.unflatten(theta.astype(np.float64), shapes)
    ref = CN.forward(params, CN.net_input(_bf16_round(u0).reshape(B, H, Wd), _bf16_round(lognu)))
    rel = np.linalg.norm(corr - ref) / np.linalg.norm(ref)
    assert rel < 3e-2, rel


def test_gradients_match_oracle():
    net, shapes, theta, u0, lognu, target = _setup(seed=2)
    B, Ns = u0.shape
    tgt = torch.as_tensor(target, dtype=torch.float32).to(torch.bfloat16).cuda().contiguous()
    with net:
        loss, g = pit.pit_net_gradients(net, torch.as_tensor(u0, device="cuda"), lognu, tgt)
    params = CN.unflatten(theta.astype(np.float64), shapes)
    inp = CN.net_input(_bf16_round(u0).reshape(B, net.shape.height, net.shape.width), _bf16_round(lognu))
    lref, grads = CN.loss_and_grad(params, inp, tgt.float().cpu().numpy().astype(np.float64))
    assert abs(loss - lref) <= 3e-2 * lref
    # layer by layer: weights and biases
    o = 0
    for (Wr, br) in grads:
        for ref in (Wr.ravel(), br.ravel()):
            got = g[o:o + ref.size].astype(np.float64)
            o += ref.size
            cos = got @ ref / (np.linalg.norm(got) * np.linalg.norm(ref) + 1e-300)
            rel = np.linalg.norm(got - ref) / (np.linalg.norm(ref) + 1e-300)
            assert cos > 0.995 and rel < 0.1, (cos, rel)
    assert o == g.size


def test_untrained_network_returns_the_plain_guess():
    net = pit.pit_net_create(8, 8, 16, 16, 1, max_batch=2, seed=3)
    with net:
        u0 = torch.randn((2, 64), dtype=torch.float64, device="cuda")
        U = torch.empty((2, 16, 64), dtype=torch.float64, device="cuda")
        pit.pit_net_guess(net, u0, np.array([-2.0, -1.5], dtype=np.float32), U)
        assert torch.equal(U, u0[:, None, :].expand(2, 16, 64))


def test_adam_training_reduces_the_loss():
    net, shapes, theta, u0, lognu, target = _setup(seed=4, B=4)
    tgt = torch.as_tensor(target, dtype=torch.float32).to(torch.bfloat16).cuda().contiguous()
    u0_d = torch.as_tensor(u0, device="cuda")
    with net:
        first = pit.pit_net_train_step(net, u0_d, lognu, tgt, 3e-3, want_loss=True)
        for _ in range(300):
            pit.pit_net_train_step(net, u0_d, lognu, tgt, 3e-3)
        last = pit.pit_net_train_step(net, u0_d, lognu, tgt, 3e-3, want_loss=True)
    assert last < 0.2 * first, (first, last)


def test_learned_guess_saves_newton_iterations():
    # small version of the learned-guess workload: train on solutions this solver
    # generates, then start Newton from the network's prediction on held-out problems
    cfg = learned.LearnedConfig(n=32, M=16, train=192, held_out=8, channels=32, blocks=2, epochs=25, batch=16)
    rep = learned.run(cfg)
    assert rep["held_out_converged_plain"] == cfg.held_out and rep["held_out_converged_learned"] == cfg.held_out
    assert rep["newton_iters_learned_mean"] < rep["newton_iters_plain_mean"], rep
    assert rep["max_rel_diff_solutions"] <= 1e-10
    # the converged solution does not depend on the start: check one against the oracle
    p = rep["check_problem"]
    Uo, _, _, _ = oracle.solve(p, tol=1e-13)
    assert np.abs(rep["check_solution"] - Uo).max() <= 1e-10 * np.abs(Uo).max()


def test_invalid_shapes_are_rejected():
    with pytest.raises(pit.PitError):
        pit.pit_net_create(8, 8, 8, 16, 1)      # levels not a multiple of 16
    with pytest.raises(pit.PitError):
        pit.pit_net_create(8, 8, 16, 24, 1)     # channels not a multiple of 16


@pytest.mark.parametrize("C,M,B,H,Wd", [(80, 144, 2, 5, 9), (16, 32, 3, 7, 130)])
def test_multi_tile_convolutions_match_oracle(C, M, B, H, Wd):
    # channel counts that split into several tensor-core tiles (80 input channels: 64 + 16;
    # 144 levels: 128 + 16 output channels) and an image row longer than one 128-pixel segment
    rng = np.random.default_rng(11)
    shapes = CN.layer_shapes(C, 1, M)
    theta = np.concatenate([np.concatenate([0.2 * rng.standard_normal(co * 9 * ci), 0.05 * rng.standard_normal(co)])
                            for co, ci in shapes]).astype(np.float32)
    u0 = rng.standard_normal((B, H * Wd))
    lognu = rng.uniform(-3, -1, B).astype(np.float32)
    target = rng.standard_normal((B, H, Wd, M)) * 0.5
    net = pit.pit_net_create(H, Wd, M, C, 1, max_batch=B, seed=1)
    pit.pit_net_set_params(net, theta)
    params = CN.unflatten(theta.astype(np.float64), shapes)
    inp = CN.net_input(_bf16_round(u0).reshape(B, H, Wd), _bf16_round(lognu))
    with net:
        U = torch.empty((B, M, H * Wd), dtype=torch.float64, device="cuda")
        pit.pit_net_guess(net, torch.as_tensor(u0, device="cuda"), lognu, U)
        corr = (U.cpu().numpy() - u0[:, None, :]).reshape(B, M, H, Wd).transpose(0, 2, 3, 1)
        tgt = torch.as_tensor(target, dtype=torch.float32).to(torch.bfloat16).cuda().contiguous()
        loss, g = pit.pit_net_gradients(net, torch.as_tensor(u0, device="cuda"), lognu, tgt)
    ref = CN.forward(params, inp)
    assert np.linalg.norm(corr - ref) / np.linalg.norm(ref) < 3e-2
    lref, grads = CN.loss_and_grad(params, inp, tgt.float().cpu().numpy().astype(np.float64))
    o = 0
    for (Wr, br) in grads:
        for ref_g in (Wr.ravel(), br.ravel()):
            got = g[o:o + ref_g.size].astype(np.float64)
            o += ref_g.size
            cos = got @ ref_g / (np.linalg.norm(got) * np.linalg.norm(ref_g) + 1e-300)
            assert cos > 0.995, cos
