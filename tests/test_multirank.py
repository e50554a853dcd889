"""The N > 1 path of bench.py on CPU: two gloo ranks (127.0.0.1), each with its own shard of
workload seeds, a barrier and a max-over-ranks of the timing -- the only collective traffic; the
evaluations themselves are independent (replicas, weak scaling). No GPU is used."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    w, r, local = bench.dist_setup()
    bench.barrier(w)
    seeds = bench.shard_seeds(r, 3)
    slowest = bench.max_over_ranks(float(10 + r), w)
    out.put((r, w, local, seeds, slowest))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_take_the_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, s0, m0), (r1, w1, l1, s1, m1) = res
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert s0 == [0, 1, 2] and s1 == [3, 4, 5]          # disjoint shards, weak scaling
    assert m0 == m1 == 11.0                              # every rank sees the slowest rank's time
