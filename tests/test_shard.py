"""Sharding one search by lexicographic rank range (host logic, CPU): the
ranges cover every combination with sizes within one, and merging the exact
top-N lists of disjoint ranges gives the global top-N.  The per-range lists
come from the oracle here; on the GPU they come from fc_search_range."""
import math
import os
import socket

import numpy as np
import pytest

import oracle
from synth import make_dataset


def _ranked_oracle_list(ds, k):
    """Every combination, ordered by (MI desc, rank asc), with its rank."""
    from paper_2201_03331_gb300 import fc_rank
    total = math.comb(ds.S, k)
    idx, sc, _ = oracle.search(ds.genotypes, ds.phenotype, k, total)
    ranks = np.array([fc_rank(ds.S, k, c) for c in idx], dtype=np.int64)
    return np.asarray(idx, dtype=np.uint32), np.asarray(sc), ranks


def _shard_list(idx, sc, ranks, r0, r1, top_n):
    keep = np.nonzero((ranks >= r0) & (ranks < r1))[0][:top_n]
    return idx[keep], sc[keep]


@pytest.mark.parametrize("total,shards", [(0, 3), (1, 4), (10, 3), (166167000, 8), (7052158645806, 522)])
def test_shard_ranges_cover_and_balance(total, shards):
    from paper_2201_03331_gb300.shard import balance_percent, shard_ranges
    r = shard_ranges(total, shards)
    assert r[0][0] == 0 and r[-1][1] == total
    assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
    sizes = [e - b for b, e in r]
    assert max(sizes) - min(sizes) <= 1
    if total >= shards:
        # Rank ranges are balanced to within one combination, far below the
        # paper's prefix distribution (under 3 %).
        assert balance_percent(sizes) <= 100.0 * shards / total + 1e-9


@pytest.mark.parametrize("k,shards,top_n", [(2, 3, 10), (3, 4, 25), (3, 7, 5), (4, 2, 40)])
def test_merge_of_range_lists_is_the_global_list(k, shards, top_n):
    from paper_2201_03331_gb300.shard import merge_shard_lists, shard_ranges
    ds = make_dataset("sh", seed=950 + k, S=12, cases=60, controls=50, k=k, top_n=top_n)
    idx, sc, ranks = _ranked_oracle_list(ds, k)
    lists = [_shard_list(idx, sc, ranks, r0, r1, top_n) for r0, r1 in shard_ranges(math.comb(ds.S, k), shards)]
    m_idx, m_sc = merge_shard_lists(ds.S, k, lists, top_n)
    assert np.array_equal(m_idx, idx[:top_n])
    assert np.array_equal(m_sc, sc[:top_n])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2201_03331_gb300.shard import gather_and_merge, shard_ranges
    k, top_n = 3, 20
    ds = make_dataset("shd", seed=960, S=11, cases=40, controls=45, k=k, top_n=top_n)
    idx, sc, ranks = _ranked_oracle_list(ds, k)
    r0, r1 = shard_ranges(math.comb(ds.S, k), world)[rank]
    local = _shard_list(idx, sc, ranks, r0, r1, top_n)
    merged = gather_and_merge(ds.S, k, local, top_n, dist)
    if rank == 0:
        out["ok"] = bool(np.array_equal(merged[0], idx[:top_n]) and np.array_equal(merged[1], sc[:top_n]))
    else:
        out[f"none{rank}"] = merged is None
    dist.destroy_process_group()


def test_two_rank_gather_and_merge():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res == {"ok": True, "none1": True}
