"""The multi-rank path of bench.py on CPU (gloo, world size 2): ranks run
disjoint histories and the timed region is the slowest rank's."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = 10.0 * (rank + 1)  # rank 1 is the slow one
    dist.barrier()
    got = bench.max_over_ranks(local, dist, "cpu")
    seeds = [bench.rank_seed(rank, i) for i in range(5)]
    q.put((rank, got, seeds))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_disjoint_seeds():
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
    by_rank = {r: (got, seeds) for r, got, seeds in out}
    assert by_rank[0][0] == by_rank[1][0] == 20.0
    assert not set(by_rank[0][1]) & set(by_rank[1][1])


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
