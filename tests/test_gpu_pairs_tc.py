"""Order-2 tensor-core path (tcgen05 0/1 e4m3 contraction + fused epilogue)
against the CPU oracle and against the prefix-table POPC sweep."""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from synth import make_config, make_dataset
from tests.parity_util import assert_topn_equal

pytestmark = pytest.mark.gpu


def fp32_bound(k, M):
    u = 2.0 ** -24
    return 2.0 * u * (2.0 * math.log(max(M, 2)) + (2.0 * 3 ** k + 6.0) * math.log(2.0))


@pytest.fixture(scope="module")
def fc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2201_03331_gb300 as fcm
    from paper_2201_03331_gb300 import build
    build.build()
    return fcm


@pytest.fixture
def path(monkeypatch):
    def set_path(p):
        monkeypatch.setenv("FC_PAIRS_PATH", p)
    return set_path


@pytest.mark.parametrize("S,cases,controls,seed", [(70, 100, 60, 1), (200, 437, 563, 2), (130, 1, 300, 3)])
def test_dense_tables_exact(fc, S, cases, controls, seed):
    ds = make_dataset("tc", seed=300 + seed, S=S, cases=cases, controls=controls, k=2, top_n=5)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    _, tab = fc.fc_pairs_dense(h, scores=False, tables=True)
    combos = np.array(list(itertools.combinations(range(S), 2)), dtype=np.uint32)
    ref = oracle.tables(ds.genotypes, ds.phenotype, 2, combos)
    got = tab[combos[:, 0], combos[:, 1]]
    bad = np.nonzero(np.any(got != ref, axis=(1, 2)))[0]
    assert len(bad) == 0, (len(bad), combos[bad[:5]], got[bad[:1]], ref[bad[:1]])
    # Entries with i >= j stay zero.
    low = np.tril_indices(S)
    assert not tab[low].any()


def test_dense_scores_within_fp32_bound(fc):
    ds = make_dataset("tcs", seed=310, S=260, cases=1500, controls=1711, k=2, top_n=5, planted=(9, 200))
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    sc, _ = fc.fc_pairs_dense(h, scores=True, tables=False)
    combos = np.array(list(itertools.combinations(range(ds.S), 2)), dtype=np.uint32)
    ref = oracle.mi(oracle.tables(ds.genotypes, ds.phenotype, 2, combos), 2)
    got = sc[combos[:, 0], combos[:, 1]].astype(np.float64)
    assert np.abs(got - ref).max() <= fp32_bound(2, ds.M)


@pytest.mark.parametrize("S,cases,controls,top_n", [(300, 900, 1100, 100), (1100, 1000, 1000, 50)])
def test_search_tc_matches_oracle(fc, path, S, cases, controls, top_n):
    path("tc")
    ds = make_dataset("tcsearch", seed=320 + S, S=S, cases=cases, controls=controls, k=2, top_n=top_n,
                      planted=(13, S - 7))
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    g_idx, g_s = fc.fc_search(h, 2, top_n)
    assert fc.fc_last_search_kind(h) == 2
    o_idx, o_s, _ = oracle.search(ds.genotypes, ds.phenotype, 2, top_n)

    def score_of(c):
        return float(oracle.mi(oracle.tables(ds.genotypes, ds.phenotype, 2, [c]), 2)[0])
    assert_topn_equal(g_idx, g_s, o_idx, o_s, score_of)
    assert tuple(g_idx[0]) == (13, S - 7)


def test_tc_and_popc_paths_agree(fc, path):
    ds = make_dataset("tcpop", seed=330, S=2500, cases=2048, controls=2048, k=2, top_n=300,
                      planted=(100, 2400), maf_range=(0.01, 0.5))
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    path("tc")
    a = fc.fc_search(h, 2, 300)
    assert fc.fc_last_search_kind(h) == 2
    path("popc")
    b = fc.fc_search(h, 2, 300)
    assert fc.fc_last_search_kind(h) in (1, 3)   # a prefix-table sweep
    assert np.array_equal(a[0], b[0])
    np.testing.assert_allclose(a[1], b[1], rtol=1e-12)


def test_all_pairs_full_size(fc, path):
    """40,000 SNPs x 8,192 samples, top 1,000 on the tensor-core path: the
    returned tables are exact, scores match the FP64 oracle, the planted
    pair ranks first, no sampled pair scores above the cut, and the POPC
    sweep returns the same list."""
    ds = make_config("C3")
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    path("tc")
    g_idx, g_s = fc.fc_search(h, 2, ds.top_n)
    assert fc.fc_last_search_kind(h) == 2
    assert len(g_s) == ds.top_n
    o_tab = oracle.tables(ds.genotypes, ds.phenotype, 2, g_idx)
    assert np.array_equal(fc.fc_tables(h, 2, g_idx), o_tab)
    np.testing.assert_allclose(g_s, oracle.mi(o_tab, 2), rtol=1e-6, atol=1e-12)
    assert tuple(g_idx[0]) == tuple(ds.planted)
    rng = np.random.default_rng(5)
    i = rng.integers(0, ds.S, 60000)
    j = rng.integers(0, ds.S, 60000)
    keep = i != j
    pairs = np.sort(np.stack([i[keep], j[keep]], axis=1), axis=1).astype(np.uint32)
    s = oracle.mi(oracle.tables(ds.genotypes, ds.phenotype, 2, pairs), 2)
    returned = {tuple(int(x) for x in r) for r in g_idx}
    for c, v in zip(pairs, s):
        if tuple(int(x) for x in c) not in returned:
            assert v <= g_s[-1] * (1 + 1e-12)
    path("popc")
    p_idx, p_s = fc.fc_search(h, 2, ds.top_n)
    assert np.array_equal(p_idx, g_idx)
    np.testing.assert_allclose(p_s, g_s, rtol=1e-12)


def test_bounded_wait_runs_out_and_the_handle_recovers(fc, path, monkeypatch):
    """Failure detection on the device: every mbarrier wait of the
    tensor-core kernel has a time budget.  FC_TEST_WAIT_TICKS shrinks the
    budget of the pipeline waits to a few hundred clock ticks, so that they
    run out on the first tile; the kernel then raises its abort flag, lets
    its copies and MMAs finish (the drain waits keep the full budget), frees
    TMEM and returns, and the search reports FC_ETIMEOUT.  The next search on
    the same handle, with the normal budget, matches the oracle."""
    ds = make_dataset("tmo", seed=330, S=300, cases=1100, controls=1237, k=2, top_n=20, planted=(30, 250))
    path("tc")
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    monkeypatch.setenv("FC_TEST_WAIT_TICKS", "200")
    with pytest.raises(fc.FiunchoError) as e:
        fc.fc_search(h, 2, 20)
    assert e.value.status == fc.FC_ETIMEOUT
    assert fc.fc_last_search_kind(h) == 2
    monkeypatch.delenv("FC_TEST_WAIT_TICKS")
    idx, s = fc.fc_search(h, 2, 20)
    assert fc.fc_last_search_kind(h) == 2
    o_idx, o_s, _ = oracle.search(ds.genotypes, ds.phenotype, 2, 20)

    def score_of(c):
        return float(oracle.mi(oracle.tables(ds.genotypes, ds.phenotype, 2, [c]), 2)[0])
    assert_topn_equal(idx, s, o_idx, o_s, score_of)
    assert tuple(idx[0]) == (30, 250)
