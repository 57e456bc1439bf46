"""The multi-rank path of bench.py on the CPU: world size 2 over gloo (the
replicas share no data; the job time is the slowest rank's and counts add)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench.dist_env()
        mx = bench.all_reduce_value(10.0 * (rank + 1), "max")
        sm = bench.all_reduce_value(rank + 1.5, "sum")
        out.put((rank, r, w, lr, mx, sm))
    finally:
        dist.destroy_process_group()


def test_two_ranks_reduce_to_the_job_values():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(k, 2, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, r, w, lr, mx, sm in got:
        assert (r, w, lr) == (rank, 2, rank)
        assert mx == 20.0 and sm == 4.0


def test_single_rank_returns_the_local_value():
    import bench
    assert not dist.is_initialized()
    assert bench.all_reduce_value(3.25, "max") == 3.25
    assert bench.all_reduce_value(3.25, "sum") == 3.25
