"""The N > 1 bench path on CPU: two gloo ranks, each with its own seeded structure (weak scaling, no data
collective), the job time taken as the max over ranks.  The per-rank solve is the CPU oracle here (test
infrastructure), so no GPU is needed."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch
    import bench
    from fetirp_gen import config
    from oracle.direct import direct
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    prob = config("c1", seed=bench.rank_seed(0, r))
    _, lam, _, _ = direct(prob)
    local_ms = 10.0 + 5.0 * r        # stand-in step times: rank 1 is the slow one

    def reduce_max(x):
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    value, ms = bench.job_throughput(local_ms, 4, w, reduce_max)
    q.put((r, float(np.linalg.norm(lam)), value, ms, float(np.sum(prob.f_nodal))))
    dist.destroy_process_group()


def test_two_ranks_weak_scaling_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, n0, v0, ms0, f0), (r1, n1, v1, ms1, f1) = out
    assert (r0, r1) == (0, 1)
    assert f0 != f1 and n0 != n1          # independent structures (different seeded loads)
    assert ms0 == ms1 == pytest.approx(15.0 / 4)      # max over ranks
    assert v0 == v1 == pytest.approx(2 * 4 / 0.015)   # whole-job solves/s
