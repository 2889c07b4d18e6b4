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


@pytest.mark.parametrize("slab_mb,enc", [(None, None), ("20", None), (None, "0"), ("20", "0")])
def test_order3_tensor_core_ranges(fc, monkeypatch, slab_mb, enc):
    """Rank ranges on the order-3 tensor-core path (one slab, and four slabs
    of pair rows; both forms of the kernel): each range list is the exact
    top-N of its combinations, and the shards merge to the whole search."""
    from paper_2201_03331_gb300.shard import merge_shard_lists, search_shard
    monkeypatch.setenv("FC_TRIPLES_PATH", "tc")
    if slab_mb:
        monkeypatch.setenv("FC_TRIPLES_SLAB_MB", slab_mb)
    if enc:
        monkeypatch.setenv("FC_TRIPLES_ENC", enc)
    ds = make_dataset("rng3", seed=975, S=130, cases=600, controls=700, k=3, top_n=25, planted=(9, 64, 121))
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    full = fc.fc_search(h, 3, 25)
    assert fc.fc_last_search_kind(h) == 6
    for r0, r1 in [(5, 50), (1000, 9000), (150000, 150001), (300000, math.comb(130, 3))]:
        idx, sc = fc.fc_search_range(h, 3, 25, r0, r1)
        assert fc.fc_last_search_kind(h) == 6
        combos = np.array([fc.fc_unrank(ds.S, 3, r) for r in range(r0, r1)], dtype=np.uint32)
        mi = oracle.mi(oracle.tables(ds.genotypes, ds.phenotype, 3, combos), 3)
        order = sorted(range(r1 - r0), key=lambda i: (-mi[i], i))[:25]
        assert np.array_equal(idx, combos[order]), (r0, r1)
        np.testing.assert_allclose(sc, mi[order], rtol=1e-6)
    lists = [search_shard(h, 3, 25, s, 3) for s in range(3)]
    m_idx, m_sc = merge_shard_lists(ds.S, 3, lists, 25)
    assert np.array_equal(m_idx, full[0])
    np.testing.assert_allclose(m_sc, full[1], rtol=1e-12)
    assert tuple(full[0][0]) == (9, 64, 121)


def test_order2_tensor_core_ranges(fc, monkeypatch):
    """Rank ranges on the order-2 tensor-core path: the tiles of the range's
    row blocks, pairs outside the range dropped in the epilogue."""
    from paper_2201_03331_gb300.shard import merge_shard_lists, search_shard
    monkeypatch.setenv("FC_PAIRS_PATH", "tc")
    ds = make_dataset("rng2", seed=976, S=300, cases=900, controls=1100, k=2, top_n=40, planted=(17, 250))
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    full = fc.fc_search(h, 2, 40)
    assert fc.fc_last_search_kind(h) == 2
    total = math.comb(300, 2)
    for r0, r1 in [(5, 50), (1000, 9000), (20000, 20001), (44000, total)]:
        idx, sc = fc.fc_search_range(h, 2, 40, r0, r1)
        assert fc.fc_last_search_kind(h) == 2
        combos = np.array([fc.fc_unrank(ds.S, 2, r) for r in range(r0, r1)], dtype=np.uint32)
        mi = oracle.mi(oracle.tables(ds.genotypes, ds.phenotype, 2, combos), 2)
        order = sorted(range(r1 - r0), key=lambda i: (-mi[i], i))[:40]
        assert np.array_equal(idx, combos[order]), (r0, r1)
        np.testing.assert_allclose(sc, mi[order], rtol=1e-6)
    lists = [search_shard(h, 2, 40, s, 4) for s in range(4)]
    m_idx, m_sc = merge_shard_lists(ds.S, 2, lists, 40)
    assert np.array_equal(m_idx, full[0])
    np.testing.assert_allclose(m_sc, full[1], rtol=1e-12)
    assert tuple(full[0][0]) == (17, 250)


@pytest.mark.parametrize("k,S,seed", [(4, 40, 1), (5, 24, 2), (6, 20, 3)])
def test_high_order_tensor_core_ranges(fc, monkeypatch, k, S, seed):
    """Rank ranges on the orders 4-6 tensor-core path: the left blocks whose
    tuples start combinations in the range, the rest dropped in the
    epilogue."""
    from paper_2201_03331_gb300.shard import merge_shard_lists, search_shard
    monkeypatch.setenv("FC_QUADS_PATH", "tc")
    ds = make_dataset("rngq", seed=980 + seed, S=S, cases=500, controls=620, k=k, top_n=30)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    full = fc.fc_search(h, k, 30)
    assert fc.fc_last_search_kind(h) == 7
    total = math.comb(S, k)
    for r0, r1 in [(0, 40), (777, 5555), (total // 2, total // 2 + 1), (total - 3000, total)]:
        idx, sc = fc.fc_search_range(h, k, 30, r0, r1)
        assert fc.fc_last_search_kind(h) == 7
        combos = np.array([fc.fc_unrank(S, k, r) for r in range(r0, r1)], dtype=np.uint32)
        mi = oracle.mi(oracle.tables(ds.genotypes, ds.phenotype, k, combos), k)
        order = sorted(range(r1 - r0), key=lambda i: (-mi[i], i))[:30]
        assert np.array_equal(idx, combos[order]), (r0, r1)
        np.testing.assert_allclose(sc, mi[order], rtol=1e-6)
    lists = [search_shard(h, k, 30, s, 3) for s in range(3)]
    m_idx, m_sc = merge_shard_lists(S, k, lists, 30)
    assert np.array_equal(m_idx, full[0])
    np.testing.assert_allclose(m_sc, full[1], rtol=1e-12)
