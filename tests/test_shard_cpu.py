"""Sharding of the batched sweep over GPUs (host logic, CPU only): the
longest-processing-time-first partition, and two gloo ranks that compute
their shares independently, as bench.py --workload batch does under
torchrun, and together cover every simulation exactly once."""
import itertools
import os
import socket
import sys

import numpy as np
import pytest

from paper_2106_12485_gb300 import workloads as W
from synthetic import plasma as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def brute_force_makespan(costs, n_parts):
    best = None
    for assign in itertools.product(range(n_parts), repeat=len(costs)):
        loads = [0] * n_parts
        for c, a in zip(costs, assign):
            loads[a] += c
        best = max(loads) if best is None else min(best, max(loads))
    return best


def test_lpt_is_a_partition_and_balanced():
    costs = W.batch_costs(P.batch_specs(256))
    for n in (1, 2, 3, 4, 8):
        parts = W.lpt_partition(costs, n)
        assert len(parts) == n
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(256))
        loads = [sum(costs[i] for i in p) for p in parts]
        # LPT: no worker carries more than the lightest one plus one job
        assert max(loads) - min(loads) <= max(costs)
        assert parts == W.lpt_partition(costs, n)      # deterministic


def test_lpt_small_cases():
    # the textbook case where LPT is not optimal: 4/3 bound
    costs = [3, 3, 2, 2, 2]
    parts = W.lpt_partition(costs, 2)
    loads = sorted(sum(costs[i] for i in p) for p in parts)
    assert loads == [5, 7]
    assert brute_force_makespan(costs, 2) == 6
    assert max(loads) <= 4 / 3 * brute_force_makespan(costs, 2)
    # random small instances against the brute-force optimum
    rng = np.random.default_rng(5)
    for _ in range(30):
        m = int(rng.integers(1, 4))
        cs = [int(v) for v in rng.integers(1, 50, size=int(rng.integers(1, 8)))]
        parts = W.lpt_partition(cs, m)
        mk = max(sum(cs[i] for i in p) for p in parts)
        opt = brute_force_makespan(cs, m)
        assert opt <= mk <= (4 / 3 - 1 / (3 * m)) * opt + 1e-9
    assert W.lpt_partition([], 3) == [[], [], []]
    with pytest.raises(ValueError):
        W.lpt_partition([1], 0)


def test_batch_particle_counts_match_the_generators():
    for spec in P.batch_specs(6):
        k = spec["ppc_side"]
        if spec["kind"] == "thermal":
            ld = P.plasma_load(spec["nx"], spec["ny"], k, k, u_th=(0.1,) * 3)
            n = len(ld["x"])
        else:
            n = sum(len(ld["x"]) for ld in P.two_clouds(
                spec["nx"], spec["ny"], k, k, drift=spec["drift"],
                u_th=spec["u_th"]))
        assert W.batch_particles(spec) == n


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
    import torch
    import torch.distributed as dist
    from paper_2106_12485_gb300 import workloads as W2
    from synthetic import plasma as P2
    r, w = bench.dist_init(world)
    specs = P2.batch_specs(256)
    costs = W2.batch_costs(specs)
    mine = W2.lpt_partition(costs, w)[r]
    # gather every rank's share (test only: the benchmark exchanges nothing)
    t = torch.full((256,), -1, dtype=torch.int64)
    t[:len(mine)] = torch.tensor(mine, dtype=torch.int64)
    out = [torch.zeros_like(t) for _ in range(w)]
    dist.all_gather(out, t)
    n_mine = sum(W2.batch_particles(specs[i]) for i in mine)
    total = bench.all_sum(float(n_mine), w)
    q.put((r, [o[o >= 0].tolist() for o in out], n_mine, total))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_the_batch():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, 2, port, q))
             for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shares = res[0][1]
    assert res[1][1] == shares                    # both ranks agree
    assert sorted(shares[0] + shares[1]) == list(range(256))
    specs = P.batch_specs(256)
    n_all = sum(W.batch_particles(s) for s in specs)
    assert res[0][3] == res[1][3] == float(n_all)
    assert res[0][2] + res[1][2] == n_all
    assert abs(res[0][2] - res[1][2]) < 0.05 * n_all
