"""Multi-process host logic of bench.py on CPU (gloo, world size 2): every
rank runs its own data set; only step times are reduced (max over ranks)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, w, local = bench.dist_info()
    assert (r, w, local) == (rank, world, rank)
    group = bench.init_group(w)
    # Rank 1 is slower; the job time is the slower rank's.
    local_ms = 100.0 if rank == 0 else 250.0
    value, ms = bench.aggregate(group, w, 1000, 5, local_ms)
    bench.barrier(group)
    out[rank] = (value, ms)
    dist.destroy_process_group()


def test_two_rank_aggregation_uses_the_slowest_rank():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        value, ms = res[rank]
        assert ms == pytest.approx(250.0 / 5)
        assert value == pytest.approx(2 * 1000 * 5 / 0.25)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.init_group(1) is None
    value, ms = bench.aggregate(None, 1, 10, 2, 40.0)
    assert value == pytest.approx(10 * 2 / 0.04) and ms == pytest.approx(20.0)
