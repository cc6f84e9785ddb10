"""The multi-process path of bench.py on CPU: world_size 2 over gloo.

bench.py --gpus N runs N independent replicas (one reservoir per rank, no
collective on the data path); only the timing is reduced (max over ranks) and
the node-updates are summed.  This exercises that logic with real gloo ranks."""
import os
import socket

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
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert bench.dist_env() == (rank, world, rank)
    seed = bench.replica_seed(rank)

    def reduce_max(vals):
        t = torch.tensor(vals, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return [float(x) for x in t]

    # rank r "took" 100 + 50 r ms for 1e6 node-updates
    value, e2e, ms, updates = bench.combine_ranks(100.0 + 50.0 * rank, 0.2 + 0.1 * rank, 1e6,
                                                  world, reduce_max)
    seeds = [None] * world
    dist.all_gather_object(seeds, seed)
    out[rank] = (value, e2e, ms, updates, tuple(seeds))
    dist.destroy_process_group()


def test_two_replica_ranks_over_gloo():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(2):
        value, e2e, ms, updates, seeds = res[r]
        assert ms == 150.0 and updates == 2e6            # slowest rank, summed work
        assert value == pytest.approx(2e6 / 0.150)
        assert e2e == pytest.approx(2e6 / 0.3)
        assert seeds == (0, 1)                           # independent replicas
