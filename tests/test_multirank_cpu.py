"""The benchmark's multi-GPU path shards OCPs across ranks with no data exchange; the only
collective is the max over ranks of the timed region.  Checked here with world_size-2 gloo
process groups on the CPU."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w = bench.workload(rank)
    slowest = bench.max_over_ranks(1.0 + rank)          # rank r took 1 + r seconds
    q.put((rank, slowest, float(w.x_s[0, 2]), bench.throughput(world, 4, slowest)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_and_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, a0, v0), (r1, s1, a1, v1) = res
    assert s0 == s1 == 2.0                 # both ranks report the slowest rank's time
    assert a0 != a1                        # each rank drew its own OCPs
    assert v0 == v1 == 2 * 256 * 4 / 2.0   # all ranks' OCPs over the slowest time


def test_single_process_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
