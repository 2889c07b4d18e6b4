"""Order-3 tensor-core path (tcgen05 contraction of 0/1 pair rows with SNP
rows, inclusion-exclusion epilogue) against the CPU oracle and against the
prefix-table POPC sweep."""
import itertools
import math

import numpy as np
import pytest

import oracle
from synth import make_config, make_dataset
from tests.parity_util import assert_topn_equal

pytestmark = pytest.mark.gpu


def fp32_bound(k, M):
    """The library's window: twice the larger of the sweep's bound and the
    order-3 tensor-core epilogue's u (7 ln M + 37 ln 2), whose n log2 n terms
    come from the hardware logarithm."""
    u = 2.0 ** -24
    lm = math.log(max(M, 2))
    sweep = u * (2.0 * lm + (2.0 * 3 ** k + 6.0) * math.log(2.0))
    return 2.0 * max(sweep, u * (7.0 * lm + 37.0 * math.log(2.0)))


@pytest.fixture(scope="module")
def fc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2201_03331_gb300 as fcm
    from paper_2201_03331_gb300 import build
    build.build()
    return fcm


@pytest.fixture(params=["1", "0"], ids=["one-accumulator", "per-class"])
def form(request, monkeypatch):
    """Both forms of the kernel: one accumulator n_case + 4096 n_ctrl (the
    default while both classes have at most 4095 samples) and one
    accumulator per class (FC_TRIPLES_ENC=0, the form for larger classes)."""
    if request.param == "0":
        monkeypatch.setenv("FC_TRIPLES_ENC", "0")
    else:
        monkeypatch.delenv("FC_TRIPLES_ENC", raising=False)
    return int(request.param)


@pytest.fixture
def path(monkeypatch):
    def set_path(p):
        monkeypatch.setenv("FC_TRIPLES_PATH", p)
    return set_path


def all_triples(S):
    return np.array(list(itertools.combinations(range(S), 3)), dtype=np.uint32)


@pytest.mark.parametrize("S,cases,controls,seed", [(3, 40, 50, 1), (33, 700, 650, 2), (70, 129, 1000, 3),
                                                   (100, 1500, 2100, 4), (131, 1, 300, 5), (97, 300, 1, 6)])
def test_dense_tables_exact(fc, form, S, cases, controls, seed):
    """Every combination's 27-cell table, for SNP counts that are not
    multiples of the 32-pair and 64-SNP blocks and ragged sample counts."""
    ds = make_dataset("t3", seed=700 + seed, S=S, cases=cases, controls=controls, k=3, top_n=5)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    assert fc.fc_triples_form(h) == form
    _, tab = fc.fc_triples_dense(h, scores=False, tables=True)
    ref = oracle.tables(ds.genotypes, ds.phenotype, 3, all_triples(S))
    bad = np.nonzero(np.any(tab != ref, axis=(1, 2)))[0]
    assert len(bad) == 0, (len(bad), all_triples(S)[bad[:5]], tab[bad[:1]], ref[bad[:1]])


def test_dense_tables_several_slabs(fc, form, monkeypatch):
    """A slab capacity of 1 MiB forces one slab per few first SNPs; the
    tables are the same."""
    monkeypatch.setenv("FC_TRIPLES_SLAB_MB", "1")
    ds = make_dataset("t3s", seed=720, S=90, cases=1100, controls=900, k=3, top_n=5)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    _, tab = fc.fc_triples_dense(h, scores=False, tables=True)
    ref = oracle.tables(ds.genotypes, ds.phenotype, 3, all_triples(90))
    assert np.array_equal(tab, ref)


def test_dense_tables_many_sample_chunks(fc, form):
    """Classes of 4,100 and 3,001 samples (33 and 24 chunks of 128 samples,
    both ragged): the pair rows formed on chip for every chunk give the
    exact tables."""
    ds = make_dataset("t3k", seed=721, S=70, cases=4100, controls=3001, k=3, top_n=5)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    _, tab = fc.fc_triples_dense(h, scores=False, tables=True)
    ref = oracle.tables(ds.genotypes, ds.phenotype, 3, all_triples(70))
    assert np.array_equal(tab, ref)


@pytest.mark.parametrize("cases,controls", [(4000, 90), (90, 4000)])
def test_dense_tables_large_classes_one_accumulator(fc, cases, controls):
    """The one-accumulator form near the ends of its range: n_case + 4096
    n_ctrl reaches about 3.7e5 (4,000 cases) and 1.6e7, close to 2^24
    (4,000 controls), and stays exact."""
    ds = make_dataset("t3e", seed=725 + cases, S=40, cases=cases, controls=controls, k=3, top_n=5)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    assert fc.fc_triples_form(h) == 1
    _, tab = fc.fc_triples_dense(h, scores=False, tables=True)
    assert np.array_equal(tab, oracle.tables(ds.genotypes, ds.phenotype, 3, all_triples(40)))


def test_dense_tables_one_accumulator_above_4096_samples(fc):
    """4,000 cases and 3,000 controls: both classes fit the one-accumulator
    form although the x ln x table outgrows the default candidate buffer
    (the kernel takes the shorter buffer instead)."""
    ds = make_dataset("t3g", seed=727, S=40, cases=4000, controls=3000, k=3, top_n=5)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    assert fc.fc_triples_form(h) == 1
    _, tab = fc.fc_triples_dense(h, scores=False, tables=True)
    assert np.array_equal(tab, oracle.tables(ds.genotypes, ds.phenotype, 3, all_triples(40)))


def test_search_short_buffer_and_long_lists_agree_with_sweep(fc, path):
    """A search in the one-accumulator form with the short candidate buffer
    (6,000 samples), and one whose list needs the per-class form (top 1,500:
    the operands are rebuilt), return the sweep's lists."""
    ds = make_dataset("t3h", seed=728, S=400, cases=3000, controls=3000, k=3, top_n=100,
                      planted=(21, 222, 383))
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    path("tc")
    a = fc.fc_search(h, 3, 100)
    assert fc.fc_last_search_kind(h) == 6
    a2 = fc.fc_search(h, 3, 1500)
    assert fc.fc_last_search_kind(h) == 6
    path("popc")
    b = fc.fc_search(h, 3, 100)
    b2 = fc.fc_search(h, 3, 1500)
    for x, y in ((a, b), (a2, b2)):
        assert np.array_equal(x[0], y[0])
        np.testing.assert_allclose(x[1], y[1], rtol=1e-12)
    assert tuple(a[0][0]) == (21, 222, 383)


def test_dense_tables_class_of_4096_takes_the_per_class_form(fc):
    big = make_dataset("t3f", seed=726, S=40, cases=4096, controls=100, k=3, top_n=5)
    hb = fc.fc_load(big.genotypes, big.phenotype)
    assert fc.fc_triples_form(hb) == 0
    _, tab = fc.fc_triples_dense(hb, scores=False, tables=True)
    assert np.array_equal(tab, oracle.tables(big.genotypes, big.phenotype, 3, all_triples(40)))


def test_dense_scores_within_fp32_bound(fc, form):
    ds = make_dataset("t3sc", seed=730, S=150, cases=1500, controls=1711, k=3, top_n=5, planted=(9, 70, 140))
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    sc, _ = fc.fc_triples_dense(h, scores=True, tables=False)
    ref = oracle.mi(oracle.tables(ds.genotypes, ds.phenotype, 3, all_triples(ds.S)), 3)
    assert np.abs(sc.astype(np.float64) - ref).max() <= fp32_bound(3, ds.M)


@pytest.mark.parametrize("S,cases,controls,top_n", [(130, 900, 1100, 100), (300, 2000, 1000, 60)])
def test_search_tc_matches_oracle(fc, form, path, S, cases, controls, top_n):
    path("tc")
    ds = make_dataset("t3search", seed=740 + S, S=S, cases=cases, controls=controls, k=3, top_n=top_n,
                      planted=(13, S // 2, S - 7))
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    g_idx, g_s = fc.fc_search(h, 3, top_n)
    assert fc.fc_last_search_kind(h) == 6
    o_idx, o_s, _ = oracle.search(ds.genotypes, ds.phenotype, 3, top_n)

    def score_of(c):
        return float(oracle.mi(oracle.tables(ds.genotypes, ds.phenotype, 3, [c]), 3)[0])
    assert_topn_equal(g_idx, g_s, o_idx, o_s, score_of)
    assert tuple(g_idx[0]) == (13, S // 2, S - 7)


def test_search_several_slabs_agree(fc, form, path, monkeypatch):
    ds = make_dataset("t3slab", seed=751, S=260, cases=1000, controls=1300, k=3, top_n=80,
                      planted=(3, 100, 250))
    path("tc")
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    a = fc.fc_search(h, 3, 80)
    monkeypatch.setenv("FC_TRIPLES_SLAB_MB", "2")
    h2 = fc.fc_load(ds.genotypes, ds.phenotype)
    b = fc.fc_search(h2, 3, 80)
    assert fc.fc_last_search_kind(h2) == 6
    c = fc.fc_search(h2, 3, 80)          # slabs rebuilt in turn on every search
    for x in (b, c):
        assert np.array_equal(a[0], x[0])
        np.testing.assert_allclose(a[1], x[1], rtol=1e-12)


def test_search_repeated_and_reloaded_agree(fc, path):
    ds = make_dataset("t3rep", seed=750, S=260, cases=1000, controls=1300, k=3, top_n=80,
                      planted=(3, 100, 250))
    path("tc")
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    a = fc.fc_search(h, 3, 80)
    h2 = fc.fc_load(ds.genotypes, ds.phenotype)
    b = fc.fc_search(h2, 3, 80)
    assert fc.fc_last_search_kind(h2) == 6
    c = fc.fc_search(h2, 3, 80)
    for x in (b, c):
        assert np.array_equal(a[0], x[0])
        np.testing.assert_allclose(a[1], x[1], rtol=1e-12)
    assert tuple(a[0][0]) == (3, 100, 250)


def test_tc_and_popc_paths_agree_full_size(fc, path):
    """1,000 SNPs x 4,000 samples, top 100: the tensor-core path and the
    sweep return the same list; the tables are exact and the planted triple
    ranks first."""
    ds = make_config("C2")
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    path("tc")
    a = fc.fc_search(h, 3, ds.top_n)
    assert fc.fc_last_search_kind(h) == 6
    path("popc")
    b = fc.fc_search(h, 3, ds.top_n)
    assert fc.fc_last_search_kind(h) in (1, 3, 4)
    assert np.array_equal(a[0], b[0])
    np.testing.assert_allclose(a[1], b[1], rtol=1e-12)
    assert tuple(a[0][0]) == tuple(ds.planted)
    o_tab = oracle.tables(ds.genotypes, ds.phenotype, 3, a[0])
    np.testing.assert_allclose(a[1], oracle.mi(o_tab, 3), rtol=1e-6, atol=1e-12)


def test_triples_dense_rejects_bad_inputs(fc):
    ds = make_dataset("t3bad", seed=760, S=600, cases=100, controls=100, k=3, top_n=5)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    with pytest.raises(fc.FiunchoError):
        fc.fc_triples_dense(h, scores=True)          # S > 512
    one = make_dataset("t3one", seed=761, S=20, cases=50, controls=0, k=3, top_n=5)
    h1 = fc.fc_load(one.genotypes, one.phenotype)
    with pytest.raises(fc.FiunchoError):
        fc.fc_triples_dense(h1, scores=True)         # a single class


def test_log2_approx_error_within_assumed_bound(fc):
    # The epilogue's error bound takes n ln n from the hardware base-2
    # logarithm with |lg2~(n) - log2 n| <= 2^-22 (log2 n + 1) for every
    # integer count 1 <= n <= 2^17: checked here for all of them (n = 0 is
    # taken as 1).
    n = np.arange(0, 2 ** 17 + 1, dtype=np.uint32)
    lg = fc.fc_log2_approx(n).astype(np.float64)
    exact = np.log2(np.maximum(n, 1).astype(np.float64))
    err = np.abs(lg - exact)
    assert (err <= 2.0 ** -22 * (exact + 1.0)).all(), (err / (exact + 1.0)).max()
    assert lg[0] == 0.0 and lg[1] == 0.0
