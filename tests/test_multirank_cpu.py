"""The benchmark's multi-rank logic on CPU: two gloo ranks on 127.0.0.1.
Single problems run as independent replicas and the batched workload's
instances are sharded by rank with no exchange; the job time is the maximum
over ranks."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert bench.dist_env() == (rank, rank, world)
    mine = bench.shard(512, rank, world)
    # per-rank times differ; the job time is the largest
    t = bench.max_over_ranks([1.0 + rank, 5.0 - rank], "cpu")
    out.put((rank, mine, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    import torch.multiprocessing as mp
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
    (r0, m0, t0), (r1, m1, t1) = res
    assert sorted(m0 + m1) == list(range(512)) and not set(m0) & set(m1)
    assert abs(len(m0) - len(m1)) <= 1
    assert t0 == t1 == [2.0, 5.0]


def test_single_rank_reduce_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.shard(5, 0, 1) == [0, 1, 2, 3, 4]
    assert bench.max_over_ranks([3.5, 1.25], "cpu") == [3.5, 1.25]
