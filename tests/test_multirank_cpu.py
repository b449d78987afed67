"""The N > 1 path of bench.py on CPU: two gloo ranks on 127.0.0.1 run the
same host-side code the benchmark runs under torchrun (barrier, max of the
ranks' times, sum of their units, one replica per rank with its own
generator stream, the reference arm on rank 0 only)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, w = bench.dist_init(world)
    assert (r, w) == (rank, world)
    bench.barrier(w)
    # rank r processed (r + 1) * 1000 units in (r + 1) * 10 ms
    value, ms_max, total = bench.aggregate((r + 1) * 1000.0, (r + 1) * 10.0, w)
    # the replica of each rank draws its own generator stream
    from paper_2106_12485_gb300 import workloads as W
    from synthetic import plasma as P
    cfg = W.precision_study(16, 16, ppc=(2, 2), sim_index=r)
    ld = P.plasma_load(16, 16, 2, 2, sim=cfg.sim_index, u_th=(0.1,) * 3)
    ux = dist_all_gather(ld["ux"][:8].astype(np.float64), w)
    # the reference arm: rank 0 alone would run it; other ranks return
    class A:
        pass
    args = A()
    args.gpus, args.steps, args.warmup, args.ppc = w, 1, 0, 2
    if r != 0:
        bench.reference_arm(args, r, w)     # returns at once, prints nothing
    q.put((r, value, ms_max, total, cfg.sim_index, ux))
    dist.barrier()
    dist.destroy_process_group()


def dist_all_gather(a, world):
    import torch
    import torch.distributed as dist
    t = torch.tensor(a)
    out = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(out, t)
    return [o.numpy() for o in out]


def test_two_gloo_ranks_aggregate_like_the_benchmark():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, 2, port, q))
             for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for r, value, ms_max, total, sim_index, ux in res:
        assert total == 3000.0               # 1000 + 2000 units
        assert ms_max == 20.0                # the slower rank
        assert value == pytest.approx(3000.0 / 0.020)
        assert sim_index == r
        # replicas differ (different generator streams), and every rank
        # sees the same gathered values
        assert not np.array_equal(ux[0], ux[1])
    np.testing.assert_array_equal(res[0][5][1], res[1][5][1])
