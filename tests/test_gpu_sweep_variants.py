"""The sweep's counting variants against the oracle: all 3^k cells one
extension SNP at a time (full), the 2^k cells with genotypes in {0,1} plus
exact inclusion-exclusion (ie, k = 2, 3), the cells whose extension SNP has
genotype 0 or 1 plus the prefix's own table (jr, k = 2..4), and all 3^k cells
from a (k-2)-prefix extended by SNP pairs (px, k = 4..6).  Every variant must
produce bit-identical tables and the same top list."""
import itertools
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


@pytest.fixture(params=["full", "ie", "jr", "px"])
def variant(request, monkeypatch):
    if request.param == "ie":
        monkeypatch.delenv("FC_SWEEP", raising=False)
    else:
        monkeypatch.setenv("FC_SWEEP", request.param)
    return request.param


@pytest.mark.parametrize("k,S,cases,controls", [(1, 40, 333, 170), (2, 45, 700, 650), (3, 26, 900, 1311),
                                                (4, 15, 400, 389), (3, 33, 1, 200)])
def test_sweep_tables_exact(fc, variant, k, S, cases, controls):
    ds = make_dataset("sw", seed=500 + k + S, S=S, cases=cases, controls=controls, k=k, top_n=5)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    total = math.comb(S, k)
    got = fc.fc_sweep_tables(h, k, 0, total)
    combos = np.array(list(itertools.combinations(range(S), k)), dtype=np.uint32)
    ref = oracle.tables(ds.genotypes, ds.phenotype, k, combos)
    bad = np.nonzero(np.any(got != ref, axis=(1, 2)))[0]
    assert len(bad) == 0, (variant, len(bad), combos[bad[:3]])


def test_sweep_tables_full_size_windows(fc, variant):
    ds = make_config("C2")
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    total = math.comb(ds.S, 3)
    rng = np.random.default_rng(9)
    for start in [0, int(rng.integers(0, total - 3000)), total - 2500]:
        n = min(2500, total - start)
        got = fc.fc_sweep_tables(h, 3, start, n)
        combos = np.array([fc.fc_unrank(ds.S, 3, r) for r in range(start, start + n)], dtype=np.uint32)
        assert np.array_equal(got, oracle.tables(ds.genotypes, ds.phenotype, 3, combos))


@pytest.mark.parametrize("k,S", [(2, 400), (3, 160)])
def test_ie_and_full_searches_agree(fc, monkeypatch, k, S):
    ds = make_dataset("agree", seed=520 + k, S=S, cases=2000, controls=2100, k=k, top_n=100,
                      planted=(5, 77, 150)[:k])
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    monkeypatch.setenv("FC_PAIRS_PATH", "popc")
    monkeypatch.delenv("FC_SWEEP", raising=False)
    a = fc.fc_search(h, k, 100)
    assert fc.fc_last_search_kind(h) == 3
    monkeypatch.setenv("FC_SWEEP", "full")
    b = fc.fc_search(h, k, 100)
    assert fc.fc_last_search_kind(h) == 1
    monkeypatch.setenv("FC_SWEEP", "jr")
    c = fc.fc_search(h, k, 100)
    assert fc.fc_last_search_kind(h) == 4
    for x in (b, c):
        assert np.array_equal(a[0], x[0])
        np.testing.assert_allclose(a[1], x[1], rtol=1e-12)
    assert tuple(a[0][0]) == (5, 77, 150)[:k]


def test_order4_variants_agree(fc, monkeypatch):
    ds = make_dataset("o4", seed=540, S=32, cases=1500, controls=1500, k=4, top_n=60,
                      planted=(2, 9, 20, 31))
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    monkeypatch.delenv("FC_SWEEP", raising=False)
    a = fc.fc_search(h, 4, 60)
    assert fc.fc_last_search_kind(h) == 5      # order 4 extends 2-prefixes by pairs by default
    monkeypatch.setenv("FC_SWEEP", "full")
    b = fc.fc_search(h, 4, 60)
    assert fc.fc_last_search_kind(h) == 1
    monkeypatch.setenv("FC_SWEEP", "jr")
    c = fc.fc_search(h, 4, 60)
    assert fc.fc_last_search_kind(h) == 4
    for x in (b, c):
        assert np.array_equal(a[0], x[0])
        np.testing.assert_allclose(a[1], x[1], rtol=1e-12)
    assert tuple(a[0][0]) == (2, 9, 20, 31)


def test_static_search_does_not_build_ie_tables(fc, monkeypatch):
    """fc_search_static must not allocate: on a fresh handle it uses the
    extension-restricted count, which needs no extra tables; once fc_search
    has built the inclusion-exclusion tables it uses them.  Both give the
    same result."""
    monkeypatch.delenv("FC_SWEEP", raising=False)
    ds = make_dataset("st-ie", seed=531, S=120, cases=1000, controls=1000, k=3, top_n=50)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    a = fc.fc_search_static(h, 3, 50)
    assert fc.fc_last_search_kind(h) == 4
    b = fc.fc_search(h, 3, 50)
    assert fc.fc_last_search_kind(h) == 3
    c = fc.fc_search_static(h, 3, 50)
    assert fc.fc_last_search_kind(h) == 3
    for x in (b, c):
        assert np.array_equal(a[0], x[0])
        np.testing.assert_allclose(a[1], x[1], rtol=1e-12)


# ---- orders 5 and 6: pair-extension sweep (default) and row-split sweep -------

@pytest.fixture(params=["px", "px-g1", "full"])
def hi_variant(request, monkeypatch):
    """px: pair extension with 27 counters per lane (default); px-g1: pair
    extension with 81 counters per lane; full: row-split kernel."""
    monkeypatch.delenv("FC_SWEEP", raising=False)
    monkeypatch.delenv("FC_SWEEP_CONFIG", raising=False)
    if request.param == "px-g1":
        monkeypatch.setenv("FC_SWEEP_CONFIG", "1,4,16")
    elif request.param == "full":
        monkeypatch.setenv("FC_SWEEP", "full")
    return request.param


@pytest.mark.parametrize("k,S,cases,controls", [(5, 9, 300, 211), (6, 9, 250, 199), (6, 8, 600, 700),
                                                (5, 10, 1, 90), (6, 6, 40, 33), (5, 5, 20, 0),
                                                (4, 23, 700, 1300), (5, 14, 3000, 100),
                                                (6, 8, 3000, 1100), (4, 12, 6000, 3000)])
def test_high_order_sweep_tables_exact(fc, hi_variant, monkeypatch, k, S, cases, controls):
    """Includes sample counts whose words span several prefix-table tiles."""
    ds = make_dataset("hi", seed=600 + k + S, S=S, cases=cases, controls=controls, k=k, top_n=5)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    total = math.comb(S, k)
    got = fc.fc_sweep_tables(h, k, 0, total)
    combos = np.array(list(itertools.combinations(range(S), k)), dtype=np.uint32)
    ref = oracle.tables(ds.genotypes, ds.phenotype, k, combos)
    assert np.array_equal(got, ref)
    if k >= 5:
        fc.fc_search(h, k, 3)
        assert fc.fc_last_search_kind(h) == (1 if hi_variant == "full" else 5)


@pytest.mark.parametrize("k,S", [(5, 40), (6, 24)])
def test_high_order_sweep_tables_windows(fc, hi_variant, k, S):
    """Windows that start and end inside prefix groups and cross them."""
    ds = make_dataset("hiw", seed=640 + k, S=S, cases=700, controls=900, k=k, top_n=5)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    total = math.comb(S, k)
    rng = np.random.default_rng(41 + k)
    for start in [0, int(rng.integers(1, total - 3000)), int(rng.integers(1, total - 3000)), total - 1777]:
        n = min(1777, total - start)
        got = fc.fc_sweep_tables(h, k, start, n)
        combos = np.array([fc.fc_unrank(S, k, r) for r in range(start, start + n)], dtype=np.uint32)
        assert np.array_equal(got, oracle.tables(ds.genotypes, ds.phenotype, k, combos)), start


@pytest.mark.parametrize("k,S,planted", [(5, 16, (1, 4, 8, 11, 15)), (6, 13, (0, 2, 5, 7, 9, 12))])
def test_high_order_search_matches_oracle(fc, hi_variant, k, S, planted):
    from tests.parity_util import assert_topn_equal
    ds = make_dataset("hi-s", seed=620 + k, S=S, cases=2048, controls=2048, k=k, top_n=30,
                      planted=planted)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    g_idx, g_s = fc.fc_search(h, k, 30)
    o_idx, o_s, tested = oracle.search(ds.genotypes, ds.phenotype, k, 30)
    assert tested == math.comb(S, k)

    def score_of(c):
        return float(oracle.mi(oracle.tables(ds.genotypes, ds.phenotype, k, [c]), k)[0])
    assert_topn_equal(g_idx, g_s, o_idx, o_s, score_of)
    assert tuple(g_idx[0]) == planted
