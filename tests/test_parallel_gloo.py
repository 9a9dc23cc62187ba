"""The multi-process path on CPU (gloo, world size 2): walker keys are disjoint
across ranks, the per-iteration histogram exchange sums over ranks, the job time
is the slowest rank's, and after the exchange every rank's Berg update (the
oracle's, here) gives the same weights -- so no weight broadcast is needed.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_1702_01770_gb300 import parallel
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    K = 50
    rng = np.random.default_rng(rank)
    local = rng.integers(0, 100, size=(4, K)).astype(np.int64)      # 4 jackknife blocks
    h = torch.from_numpy(local.copy())
    parallel.combine_histograms(h)
    t = parallel.max_over_ranks(float(rank + 1), torch.device("cpu"))
    lnW, g, _ = oracle.berg_update(h.sum(0).numpy().astype(float), np.zeros(K), np.zeros(K - 1), 0.1)
    out.put((rank, local, h.numpy(), t, lnW, parallel.walker_seed_base(rank, 16384)))
    dist.destroy_process_group()


def test_histogram_exchange_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=120) for _ in range(2)], key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    total = res[0][1] + res[1][1]
    assert np.array_equal(res[0][2], total) and np.array_equal(res[1][2], total)
    assert res[0][3] == res[1][3] == 2.0
    assert np.array_equal(res[0][4], res[1][4])                  # identical weights on both ranks
    assert res[0][5] == 0 and res[1][5] == 16384                 # disjoint walker keys


def test_single_process_is_a_no_op():
    from paper_1702_01770_gb300 import parallel
    h = torch.arange(10)
    assert torch.equal(parallel.combine_histograms(h.clone()), h)
    assert parallel.max_over_ranks(3.5, torch.device("cpu")) == 3.5
    assert parallel.world() == (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
                                int(os.environ.get("LOCAL_RANK", 0)))
