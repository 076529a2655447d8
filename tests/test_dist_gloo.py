"""Multi-process host logic of replica runs, on CPU with the gloo backend (world size 2):
the timed region's barrier, the maximum of the per-rank times, the whole-job value, and
the round-robin sharding of a batch of independent problems."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2406_00878_gb300 import dist as D  # noqa: E402
from paper_2406_00878_gb300 import workloads as W  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = D.env()
        D.barrier()
        # rank r "took" 10 + 5 r ms; the job takes as long as the slowest rank
        ms = D.max_over_ranks(10.0 + 5.0 * r)
        value = D.job_throughput([1000.0] * ws, ms * 1e-3)
        probs = W.batched(seed=0, count=10)
        mine = D.shard(len(probs), r, ws)
        q.put((r, ws, local, ms, value, mine, [probs[i].name for i in mine]))
        D.barrier()
    finally:
        tdist.destroy_process_group()


def test_replica_timing_and_sharding_over_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for r, (rank, ws, local, ms, value, mine, names) in enumerate(out):
        assert (rank, ws, local) == (r, world, r)
        assert ms == 15.0                      # max over ranks
        assert value == pytest.approx(2000.0 / 15e-3)
    owned = sorted(i for o in out for i in o[5])
    assert owned == list(range(10))            # every problem exactly once
    assert not set(out[0][6]) & set(out[1][6])


def test_shard_and_throughput_single_process():
    assert D.shard(7, 0, 3) == [0, 3, 6] and D.shard(7, 2, 3) == [2, 5]
    with pytest.raises(ValueError):
        D.shard(4, 3, 3)
    assert D.max_over_ranks(3.5) == 3.5       # no process group: the value itself
    assert D.job_throughput([10, 20], 2.0) == 15.0
    with pytest.raises(ValueError):
        D.job_throughput([1], 0.0)
