"""Multi-GPU path = replicas (independent structures per rank), exercised
with two gloo ranks on CPU: each rank builds its own seeded structure, the
job time is the slowest rank's (max over ranks), and the whole-job rate
counts every rank's cells."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    from paper_1410_1914_gb300 import inputs
    from paper_1410_1914_gb300.replicas import aggregate_rate, max_over_ranks, rank_seed
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ph, _, _ = inputs.make_workload("pt_cl_256", shape=(8, 8, 16), seed=rank_seed(1, rank))
        dist.barrier()
        t = max_over_ranks(0.5 + rank, dist)  # rank r "took" 0.5 + r seconds
        out[rank] = (t, aggregate_rate(ph.size * 10, world, t), ph.tobytes())
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        for p in procs:
            if p.is_alive():
                p.kill()
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        res = dict(out)
    t0, rate0, s0 = res[0]
    t1, rate1, s1 = res[1]
    assert t0 == t1 == 1.5                      # the slowest rank's time on every rank
    cells = 8 * 8 * 16
    assert rate0 == rate1 == pytest.approx(cells * 10 * 2 / 1.5)
    assert s0 != s1                             # each rank solves its own structure


def test_single_process_defaults():
    from paper_1410_1914_gb300.replicas import aggregate_rate, max_over_ranks, rank_seed
    assert max_over_ranks(3.25) == 3.25
    assert aggregate_rate(10.0, 1, 2.0) == 5.0
    assert [rank_seed(1, r) for r in range(3)] == [1, 2, 3]
    assert np.isfinite(aggregate_rate(1.0, 4, 1e-3))
