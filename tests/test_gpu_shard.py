"""fc_search_range and the rank-range sharding of one search on the GPU:
the merged lists of disjoint ranges equal fc_search's list, and a range's
list is the exact top-N of its combinations."""
import math

import numpy as np
import pytest

import oracle
from synth import make_config, make_dataset

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2201_03331_gb300 as fcm
    from paper_2201_03331_gb300 import build
    build.build()
    return fcm


@pytest.mark.parametrize("name,snps,shards", [("C2", 300, 3), ("C4", 60, 4), ("C1", None, 5)])
def test_shards_merge_to_the_full_search(fc, name, snps, shards):
    from paper_2201_03331_gb300.shard import merge_shard_lists, search_shard
    ds = make_config(name, snps)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    full = fc.fc_search(h, ds.k, ds.top_n)
    lists = [search_shard(h, ds.k, ds.top_n, s, shards) for s in range(shards)]
    m_idx, m_sc = merge_shard_lists(ds.S, ds.k, lists, ds.top_n)
    assert np.array_equal(m_idx, full[0])
    np.testing.assert_allclose(m_sc, full[1], rtol=1e-12)


def test_range_list_is_exact_top_n_of_the_range(fc):
    ds = make_dataset("rng", seed=970, S=40, cases=700, controls=650, k=3, top_n=30)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    total = math.comb(ds.S, 3)
    r0, r1 = 2000, 7000
    idx, sc = fc.fc_search_range(h, 3, 30, r0, r1)
    combos = np.array([fc.fc_unrank(ds.S, 3, r) for r in range(r0, r1)], dtype=np.uint32)
    mi = oracle.mi(oracle.tables(ds.genotypes, ds.phenotype, 3, combos), 3)
    order = sorted(range(r1 - r0), key=lambda i: (-mi[i], i))[:30]
    assert np.array_equal(idx, combos[order])
    np.testing.assert_allclose(sc, mi[order], rtol=1e-6)
    # Empty and whole ranges.
    e_idx, e_sc = fc.fc_search_range(h, 3, 30, 5, 5)
    assert len(e_sc) == 0
    w = fc.fc_search_range(h, 3, 30, 0, total)
    f = fc.fc_search(h, 3, 30)
    assert np.array_equal(w[0], f[0])
    with pytest.raises(fc.FiunchoError):
        fc.fc_search_range(h, 3, 30, 10, total + 1)
