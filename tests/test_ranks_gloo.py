"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): each rank
gets its own seed vertex (independent problems, no data-path collective) and
the timing/work aggregation takes the max of times and the sum of work."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1604_07515_gb300 import inputs
    off, col = inputs.rmat(10, seed=5)
    seed = bench.rank_seed(off, col, rank)
    mx, sm = bench.reduce_ranks([10.0 * (rank + 1)], [100.0 + rank, 1.0], world, "cpu")
    seeds = [None] * world
    dist.all_gather_object(seeds, seed)
    q.put((rank, seed, mx, sm, seeds))
    dist.destroy_process_group()


def test_two_ranks_shard_seeds_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, seed, mx, sm, seeds in out:
        assert mx == [20.0]
        assert sm == [201.0, 2.0]
        assert len(set(seeds)) == 2  # independent problems per rank
