"""Tensor-core path of orders 4-6 (tcgen05 contraction of 0/1 tuple rows
with tuple rows, all 3^k cells) against the CPU oracle and against the
pair-extension sweep."""
import itertools
import math

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
        monkeypatch.setenv("FC_QUADS_PATH", p)
    return set_path


@pytest.fixture(params=["1", "0"], ids=["one-accumulator", "per-class"])
def form(request, monkeypatch):
    """Form 1 (controls carry 64, one accumulator n_case + 4096 n_ctrl, two
    right blocks per tile) where both classes allow it, or form 0."""
    monkeypatch.setenv("FC_QUADS_ENC", request.param)
    return int(request.param)


def all_quads(S):
    return np.array(list(itertools.combinations(range(S), 4)), dtype=np.uint32)


@pytest.mark.parametrize("S,cases,controls,seed", [(4, 40, 50, 1), (13, 700, 650, 2), (30, 129, 1000, 3),
                                                   (41, 1500, 2100, 4), (26, 1, 300, 5), (19, 300, 1, 6)])
def test_dense_tables_exact(fc, form, S, cases, controls, seed):
    """Every combination's 81-cell table, for pair counts that leave partial
    blocks and ragged sample counts."""
    ds = make_dataset("q4", seed=800 + seed, S=S, cases=cases, controls=controls, k=4, top_n=5)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    _, tab = fc.fc_tuples_dense(h, 4, scores=False, tables=True)
    ref = oracle.tables(ds.genotypes, ds.phenotype, 4, all_quads(S))
    bad = np.nonzero(np.any(tab != ref, axis=(1, 2)))[0]
    assert len(bad) == 0, (len(bad), all_quads(S)[bad[:5]])


@pytest.mark.parametrize("cases,controls", [(4000, 90), (90, 4000), (4096, 300)])
def test_dense_tables_class_limits(fc, monkeypatch, cases, controls):
    """Near the ends of the one-accumulator range (n_case + 4096 n_ctrl up to
    about 1.6e7) and just past it (4,096 cases: the per-class form)."""
    monkeypatch.setenv("FC_QUADS_ENC", "1")
    ds = make_dataset("q4e", seed=840 + cases, S=14, cases=cases, controls=controls, k=4, top_n=5)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    _, tab = fc.fc_tuples_dense(h, 4, scores=False, tables=True)
    assert np.array_equal(tab, oracle.tables(ds.genotypes, ds.phenotype, 4, all_quads(14)))


def test_dense_scores_within_fp32_bound(fc):
    ds = make_dataset("q4sc", seed=830, S=48, cases=1500, controls=1711, k=4, top_n=5, planted=(3, 17, 30, 44))
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    sc, _ = fc.fc_tuples_dense(h, 4, scores=True, tables=False)
    ref = oracle.mi(oracle.tables(ds.genotypes, ds.phenotype, 4, all_quads(ds.S)), 4)
    assert np.abs(sc.astype(np.float64) - ref).max() <= fp32_bound(4, ds.M)


@pytest.mark.parametrize("S,cases,controls,top_n", [(40, 900, 1100, 100), (70, 2000, 1000, 60)])
def test_search_tc_matches_oracle(fc, form, path, S, cases, controls, top_n):
    path("tc")
    ds = make_dataset("q4search", seed=840 + S, S=S, cases=cases, controls=controls, k=4, top_n=top_n,
                      planted=(3, S // 3, S // 2, S - 5))
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    g_idx, g_s = fc.fc_search(h, 4, top_n)
    assert fc.fc_last_search_kind(h) == 7
    o_idx, o_s, _ = oracle.search(ds.genotypes, ds.phenotype, 4, top_n)

    def score_of(c):
        return float(oracle.mi(oracle.tables(ds.genotypes, ds.phenotype, 4, [c]), 4)[0])
    assert_topn_equal(g_idx, g_s, o_idx, o_s, score_of)
    assert tuple(g_idx[0]) == (3, S // 3, S // 2, S - 5)


def test_tc_and_sweep_agree_full_size(fc, path):
    """300 SNPs x 6,000 samples, top 100: the tensor-core path and the
    pair-extension sweep return the same list; the planted quadruple ranks
    first and the returned tables are exact."""
    ds = make_config("C4")
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    path("tc")
    a = fc.fc_search(h, 4, ds.top_n)
    assert fc.fc_last_search_kind(h) == 7
    path("popc")
    b = fc.fc_search(h, 4, ds.top_n)
    assert fc.fc_last_search_kind(h) == 5
    assert np.array_equal(a[0], b[0])
    np.testing.assert_allclose(a[1], b[1], rtol=1e-12)
    assert tuple(a[0][0]) == tuple(ds.planted)
    o_tab = oracle.tables(ds.genotypes, ds.phenotype, 4, a[0])
    assert np.array_equal(fc.fc_tables(h, 4, a[0]), o_tab)
    np.testing.assert_allclose(a[1], oracle.mi(o_tab, 4), rtol=1e-6, atol=1e-12)


def test_tuples_dense_rejects_bad_inputs(fc):
    ds = make_dataset("q4bad", seed=860, S=200, cases=100, controls=100, k=4, top_n=5)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    with pytest.raises(fc.FiunchoError):
        fc.fc_tuples_dense(h, 4, scores=True)       # C(200, 4) > 2^25
    one = make_dataset("q4one", seed=861, S=12, cases=50, controls=0, k=4, top_n=5)
    h1 = fc.fc_load(one.genotypes, one.phenotype)
    with pytest.raises(fc.FiunchoError):
        fc.fc_tuples_dense(h1, 4, scores=True)      # a single class
    with pytest.raises(fc.FiunchoError):
        fc.fc_tuples_dense(h1, 3, scores=True)      # order outside 4..6


# ---- orders 5 and 6 ----------------------------------------------------------

def all_k(S, k):
    return np.array(list(itertools.combinations(range(S), k)), dtype=np.uint32)


@pytest.mark.parametrize("k,S,cases,controls,seed", [(5, 5, 40, 50, 1), (5, 14, 700, 650, 2), (5, 29, 300, 290, 3),
                                                     (6, 6, 60, 41, 4), (6, 13, 129, 600, 5), (6, 20, 1, 333, 6)])
def test_high_order_dense_tables_exact(fc, form, k, S, cases, controls, seed):
    ds = make_dataset("t56", seed=870 + seed, S=S, cases=cases, controls=controls, k=k, top_n=5)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    _, tab = fc.fc_tuples_dense(h, k, scores=False, tables=True)
    ref = oracle.tables(ds.genotypes, ds.phenotype, k, all_k(S, k))
    bad = np.nonzero(np.any(tab != ref, axis=(1, 2)))[0]
    assert len(bad) == 0, (len(bad), all_k(S, k)[bad[:5]])


@pytest.mark.parametrize("k,S", [(5, 26), (6, 19)])
def test_high_order_dense_scores_within_fp32_bound(fc, k, S):
    ds = make_dataset("t56sc", seed=890 + k, S=S, cases=1024, controls=1024, k=k, top_n=5)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    sc, _ = fc.fc_tuples_dense(h, k, scores=True, tables=False)
    ref = oracle.mi(oracle.tables(ds.genotypes, ds.phenotype, k, all_k(S, k)), k)
    assert np.abs(sc.astype(np.float64) - ref).max() <= fp32_bound(k, ds.M)


@pytest.mark.parametrize("k,S,planted", [(5, 30, (2, 9, 15, 22, 29)), (6, 22, (1, 5, 9, 13, 17, 21))])
def test_high_order_search_tc_matches_oracle(fc, form, path, k, S, planted):
    path("tc")
    ds = make_dataset("t56s", seed=900 + k, S=S, cases=1024, controls=1024, k=k, top_n=40, planted=planted)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    g_idx, g_s = fc.fc_search(h, k, 40)
    assert fc.fc_last_search_kind(h) == 7
    o_idx, o_s, _ = oracle.search(ds.genotypes, ds.phenotype, k, 40)

    def score_of(c):
        return float(oracle.mi(oracle.tables(ds.genotypes, ds.phenotype, k, [c]), k)[0])
    assert_topn_equal(g_idx, g_s, o_idx, o_s, score_of)
    assert tuple(g_idx[0]) == planted


@pytest.mark.parametrize("name,S", [("P5", 70), ("P6", 44)])
def test_high_order_tc_and_sweep_agree(fc, path, name, S):
    """The order-5 and order-6 workloads cut to their first SNPs: the
    tensor-core path and the pair-extension sweep return the same list."""
    ds = make_config(name, scale_snps=S)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    path("tc")
    a = fc.fc_search(h, ds.k, ds.top_n)
    assert fc.fc_last_search_kind(h) == 7
    path("popc")
    b = fc.fc_search(h, ds.k, ds.top_n)
    assert fc.fc_last_search_kind(h) == 5
    assert np.array_equal(a[0], b[0])
    np.testing.assert_allclose(a[1], b[1], rtol=1e-12)


# ---- right operand in chunks -------------------------------------------------
# When the right tuple rows do not fit beside the left ones (the paper's
# single-node order-5 and order-6 sizes), the search builds them chunk by
# chunk and runs each chunk's tiles.  FC_TUPLES_SLAB_MB makes small cases
# take that path.

def _slab_mb(k, S, M1, M0, form, right_share):
    """Memory cap (MB) that leaves about `right_share` of the right rows beside
    the left ones: blocks of 128 rows of (words * 128 + 128) bytes, 12 left
    pairs or 4 triples per block (one tuple of each genotype combination per
    32-row quarter), right blocks in pairs in form 1."""
    LT = 3 if k == 6 else 2
    RT = k - LT
    words = -(-M1 // 128) + -(-M0 // 128)
    blk = 128 * (words * 128 + 128)
    per = {2: 12, 3: 4}
    bl = -(-math.comb(S - RT, LT) // per[LT])
    br = -(-math.comb(S - LT, RT) // per[RT])
    left, right = bl * blk, br * blk
    return int(math.ceil((left + right_share * right) / 2 ** 20)), left + right


@pytest.mark.parametrize("k,S,cases,controls,seed", [(4, 41, 1500, 2100, 11), (5, 29, 300, 290, 12),
                                                     (6, 20, 1, 333, 13)])
def test_dense_tables_exact_right_chunks(fc, form, monkeypatch, k, S, cases, controls, seed):
    mb, total = _slab_mb(k, S, cases, controls, form, 0.25)
    assert mb * 2 ** 20 < total            # the right rows cannot all stay
    monkeypatch.setenv("FC_TUPLES_SLAB_MB", str(mb))
    ds = make_dataset("q4chunk", seed=870 + seed, S=S, cases=cases, controls=controls, k=k, top_n=5)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    fc.fc_timing(h, 1)
    _, tab = fc.fc_tuples_dense(h, k, scores=False, tables=True)
    _, _, launches = fc.fc_timing(h, 0)
    assert launches >= 2 + 2 * 3           # left rows + at least three (right chunk, kernel) launches
    ref = oracle.tables(ds.genotypes, ds.phenotype, k, all_k(S, k))
    bad = np.nonzero(np.any(tab != ref, axis=(1, 2)))[0]
    assert len(bad) == 0, (len(bad), all_k(S, k)[bad[:5]])


@pytest.mark.parametrize("k,S,cases,controls,top_n", [(5, 34, 500, 420, 60), (6, 24, 300, 333, 40)])
def test_search_right_chunks_match_oracle(fc, form, path, monkeypatch, k, S, cases, controls, top_n):
    path("tc")
    mb, _ = _slab_mb(k, S, cases, controls, form, 0.2)
    monkeypatch.setenv("FC_TUPLES_SLAB_MB", str(mb))
    planted = tuple(sorted({2, S // 4, S // 3, S // 2, 2 * S // 3, S - 3}))[:k]
    ds = make_dataset("q5chunk", seed=880 + k, S=S, cases=cases, controls=controls, k=k, top_n=top_n,
                      planted=planted)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    g_idx, g_s = fc.fc_search(h, k, top_n)
    assert fc.fc_last_search_kind(h) == 7
    o_idx, o_s, _ = oracle.search(ds.genotypes, ds.phenotype, k, top_n)

    def score_of(c):
        return float(oracle.mi(oracle.tables(ds.genotypes, ds.phenotype, k, [c]), k)[0])
    assert_topn_equal(g_idx, g_s, o_idx, o_s, score_of)
    # The same search again (the right rows of the last chunk are in place),
    # and a rank range, against a handle whose right rows all fit.
    again = fc.fc_search(h, k, top_n)
    assert np.array_equal(again[0], g_idx)
    monkeypatch.delenv("FC_TUPLES_SLAB_MB")
    h1 = fc.fc_load(ds.genotypes, ds.phenotype)
    total = math.comb(S, k)
    r0, r1 = total // 3, total // 3 + total // 5
    a = fc.fc_search_range(h, k, top_n, r0, r1)
    b = fc.fc_search_range(h1, k, top_n, r0, r1)
    assert fc.fc_last_search_kind(h1) == 7
    assert np.array_equal(a[0], b[0])
    np.testing.assert_allclose(a[1], b[1], rtol=1e-12)
