"""The multi-GPU path of bench.py (replicas, one process per GPU) on CPU:
two gloo ranks check the pair sharding, the max-over-ranks step time and
the whole-job throughput.  Pairs are independent, so no exchange step
exists; the only collectives are the timing barrier and reduction."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ids = bench.rank_pair_ids(rank, 64)
        wl = bench.workload(rank, 4)  # descriptors of this rank's pairs
        gathered = [None] * world
        dist.all_gather_object(gathered, (ids, [p.pair_id for p in wl.pairs]))
        local_ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        slowest = bench.max_over_ranks(local_ms, dist)
        dist.barrier()
        q.put((rank, gathered, slowest, bench.aggregate_pairs_per_s(world, 64, 3, slowest * 3)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_pairs_and_reduce_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, slowest, value in out:
        (ids0, wl0), (ids1, wl1) = gathered
        assert sorted(ids0 + ids1) == list(range(128)) and not set(ids0) & set(ids1)
        assert wl0 == [0, 1, 2, 3] and wl1 == [4, 5, 6, 7]
        assert slowest == 15.0
        assert value == pytest.approx(2 * 64 / 15e-3)
