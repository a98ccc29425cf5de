"""The bench's multi-rank host logic on CPU: two gloo ranks (127.0.0.1), each
taking its own, distinct lattices of the workload (weak scaling), and the job
time taken as the slowest rank's -- what bench.py does under torchrun, where
the only collectives are the timing barrier and this maximum."""
import datetime
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=60))
    try:
        for name in ("temperature4096", "large16384"):
            sims, _ = bench.workload(name)
            mine = [s.seed for s in bench.rank_sims(sims, rank)]
            seeds = [None] * world
            dist.all_gather_object(seeds, mine)
            t = bench.max_over_ranks(1.0 + 0.5 * rank, dist, "cpu")
            dist.barrier()
            out.put((name, rank, seeds, t))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_distinct_lattices_and_the_slowest_time():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    results = [out.get(timeout=120) for _ in range(4)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import bench

    for name, rank, seeds, t in results:
        sims, _ = bench.workload(name)
        assert seeds[0] == [s.seed for s in sims]                   # rank 0: the workload
        assert seeds[1] == [s.seed + len(sims) for s in sims]      # rank 1: shifted
        assert not set(seeds[0]) & set(seeds[1])                  # no lattice twice
        assert t == pytest.approx(1.5)                            # the slowest rank
