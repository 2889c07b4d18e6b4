"""One exhaustive search sharded over several devices or processes.

The combinations of order k are split into contiguous lexicographic rank
ranges of equal size (to within one combination), one per shard; each shard
searches its range exactly with ``fc_search_range`` and the shards' lists are
merged by (score desc, rank asc).  The merge is exact: every member of the
global top-N is in the top-N of its own range.  This is the paper's
distribution of the combinations over processing units (Section
"Distribution strategy") with rank ranges in place of its round-robin of
(k-1)-prefixes; ``balance_percent`` is the paper's balance measure (Section
"Parallel distribution balance") for comparing the two.

Only host-side bookkeeping lives here; every combination is counted and
scored by the library's kernels.
"""
from __future__ import annotations

import math

import numpy as np

from . import _binding as _b


def shard_ranges(total: int, shards: int):
    """Contiguous rank ranges [begin, end) of sizes differing by at most one."""
    if shards < 1:
        raise ValueError("shards must be >= 1")
    return [(total * i // shards, total * (i + 1) // shards) for i in range(shards)]


def balance_percent(counts) -> float:
    """100 (max d_i - mean) / mean over the combinations d_i per unit."""
    counts = np.asarray(counts, dtype=np.float64)
    mean = counts.sum() / len(counts)
    return 100.0 * (counts.max() - mean) / mean


def merge_shard_lists(S: int, k: int, lists, top_n: int):
    """Merge per-shard ``(indices uint32[n][k], scores float64[n])`` lists of
    disjoint rank ranges into the global top ``top_n`` (score desc, rank asc)."""
    rows = []
    for idx, sc in lists:
        idx = np.asarray(idx, dtype=np.uint32).reshape(-1, k)
        for r in range(len(sc)):
            rows.append((-float(sc[r]), _b.fc_rank(S, k, idx[r]), idx[r]))
    rows.sort(key=lambda t: (t[0], t[1]))
    rows = rows[:top_n]
    out_idx = np.array([r[2] for r in rows], dtype=np.uint32).reshape(-1, k)
    out_sc = np.array([-r[0] for r in rows], dtype=np.float64)
    return out_idx, out_sc


def search_shard(h, k: int, top_n: int, shard: int, shards: int):
    """This shard's exact top-N (its rank range of C(S, k))."""
    S = _b.fc_info(h)[0]
    r0, r1 = shard_ranges(math.comb(S, k), shards)[shard]
    return _b.fc_search_range(h, k, top_n, r0, r1)


def gather_and_merge(S: int, k: int, local, top_n: int, dist, dst: int = 0):
    """Gather every rank's ``local`` list on rank ``dst`` over
    ``torch.distributed`` and merge them there (None on the other ranks)."""
    world = dist.get_world_size()
    payload = (np.asarray(local[0], dtype=np.uint32), np.asarray(local[1], dtype=np.float64))
    gathered = [None] * world if dist.get_rank() == dst else None
    dist.gather_object(payload, gathered, dst=dst)
    if dist.get_rank() != dst:
        return None
    return merge_shard_lists(S, k, gathered, top_n)


def distributed_search(h, k: int, top_n: int, dist, dst: int = 0):
    """The search of handle ``h`` sharded over the ranks of ``dist`` (each
    rank holds the same data set on its own device): the merged list on
    rank ``dst``, None elsewhere."""
    S = _b.fc_info(h)[0]
    local = search_shard(h, k, top_n, dist.get_rank(), dist.get_world_size())
    return gather_and_merge(S, k, local, top_n, dist, dst)
