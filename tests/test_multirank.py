"""The N > 1 paths on CPU with two gloo ranks: the benchmark's job time is the
slowest rank's and its value the units of all ranks over that time; request
sharding for several GPUs is a partition balanced by footprint."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local_ms = 100.0 * (rank + 1)                 # rank 1 is the slow one
        ms_max, value = bench.aggregate(local_ms, units_per_rank=1000, world=world)
        from paper_1206_1361_gb300.serve import shard_requests
        from paper_1206_1361_gb300.workloads import request_stream
        reqs = request_stream(count=50)
        mine = shard_requests(reqs, world, rank)
        out.put((rank, ms_max, value, [r.arrival for r in mine],
                 sum(r.inst.points for r in mine)))
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_and_shard():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = [out.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    for rank, ms_max, value, _, _ in got:
        assert ms_max == 200.0                        # max over ranks
        assert value == pytest.approx(2 * 1000 / 0.2)
    a, b = set(got[0][3]), set(got[1][3])
    assert not a & b and len(a) + len(b) == 50        # a partition of the stream
    pa, pb = got[0][4], got[1][4]
    assert abs(pa - pb) <= 0.2 * max(pa, pb)          # balanced by footprint
