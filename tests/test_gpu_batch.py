"""Batched persistent search (many data sets x phenotype replicates in one
graph-captured launch) against the oracle and against per-job launches."""
import math

import numpy as np
import pytest

import oracle
from synth import make_batch, make_dataset, permuted_phenotypes
from tests.parity_util import assert_topn_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2201_03331_gb300 as fcm
    from paper_2201_03331_gb300 import build
    build.build()
    return fcm


def _small_batch(seed, n, R, snp_range, sample_range, k):
    return make_batch(n_datasets=n, replicates=R, seed=seed, snp_range=snp_range,
                      sample_range=sample_range, k=k, top_n=10)


@pytest.mark.parametrize("k,snps,samples", [(3, (40, 90), (300, 1200)), (2, (60, 150), (200, 900)),
                                            (4, (20, 30), (400, 700))])
def test_batch_matches_oracle_per_job(fc, k, snps, samples):
    batch = _small_batch(50 + k, 4, 3, snps, samples, k)
    h = fc.fc_load_batch([ds.genotypes for ds, _ in batch], [ph for _, ph in batch])
    assert fc.fc_batch_info(h) == (4, 3, 12)
    idx, score, cnt = fc.fc_search_batch(h, k, 10)
    for d, (ds, ph) in enumerate(batch):
        for r in range(3):
            j = d * 3 + r
            o_idx, o_s, tested = oracle.search(ds.genotypes, ph[r], k, 10)
            assert cnt[j] == min(10, math.comb(ds.S, k)) == len(o_s)

            def score_of(c, ds=ds, ph=ph, r=r):
                return float(oracle.mi(oracle.tables(ds.genotypes, ph[r], k, [c]), k)[0])
            assert_topn_equal(idx[j, :cnt[j]], score[j, :cnt[j]], o_idx, o_s, score_of)


def test_batch_equals_per_job_launches_and_replays(fc):
    batch = _small_batch(61, 6, 4, (80, 200), (500, 3000), 3)
    h = fc.fc_load_batch([ds.genotypes for ds, _ in batch], [ph for _, ph in batch])
    a = fc.fc_search_batch(h, 3, 10)
    b = fc.fc_search_batch(h, 3, 10)   # graph replay
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    for j in range(24):
        idx, s = fc.fc_search_job(h, j, 3, 10)
        assert np.array_equal(idx, a[0][j, :len(s)])
        np.testing.assert_allclose(s, a[1][j, :len(s)], rtol=1e-12)
    # A different (k, top_n) re-plans and still agrees.
    c = fc.fc_search_batch(h, 2, 7)
    for j in (0, 5, 23):
        idx, s = fc.fc_search_job(h, j, 2, 7)
        assert np.array_equal(idx, c[0][j]) and np.allclose(s, c[1][j], rtol=1e-12)


def test_batch_uneven_and_tiny_jobs(fc):
    # One data set with exactly k SNPs (one combination), one where top_n
    # exceeds the number of combinations, one large.
    sets = [make_dataset("u0", seed=71, S=3, cases=40, controls=61, k=3, top_n=10),
            make_dataset("u1", seed=72, S=6, cases=300, controls=200, k=3, top_n=10),
            make_dataset("u2", seed=73, S=120, cases=900, controls=1300, k=3, top_n=10,
                         planted=(4, 60, 119))]
    phs = [permuted_phenotypes(ds.phenotype, 2, seed=80 + i) for i, ds in enumerate(sets)]
    h = fc.fc_load_batch([ds.genotypes for ds in sets], phs)
    idx, score, cnt = fc.fc_search_batch(h, 3, 10)
    assert cnt.tolist() == [1, 1, 10, 10, 10, 10]
    assert idx[0, 0].tolist() == [0, 1, 2]
    assert tuple(idx[4, 0]) == (4, 60, 119)     # replicate 0: the planted triple
    for j, (ds, ph) in enumerate([(s, p[r]) for s, p in zip(sets, phs) for r in range(2)]):
        o_idx, o_s, _ = oracle.search(ds.genotypes, ph, 3, 10)

        def score_of(c, ds=ds, ph=ph):
            return float(oracle.mi(oracle.tables(ds.genotypes, ph, 3, [c]), 3)[0])
        assert_topn_equal(idx[j, :cnt[j]], score[j, :cnt[j]], o_idx, o_s, score_of)


def test_batch_rejects_bad_order(fc):
    sets = [make_dataset("b0", seed=91, S=5, cases=20, controls=20, k=3, top_n=3),
            make_dataset("b1", seed=92, S=9, cases=20, controls=20, k=3, top_n=3)]
    h = fc.fc_load_batch([ds.genotypes for ds in sets], [ds.phenotype[None, :] for ds in sets])
    with pytest.raises(fc.FiunchoError) as e:
        fc.fc_search_batch(h, 6, 3)    # larger than the smallest S
    assert e.value.status == fc.FC_EINVAL
    with pytest.raises(fc.FiunchoError):
        fc.fc_search(h, 2, 3)          # a batch handle has no single data set


def test_batch_hybrid_tensor_core_jobs(fc, monkeypatch):
    """Order-3 jobs with enough SNPs for the tensor cores run on that path
    after the persistent launch; the lists equal those of the all-sweep batch
    and of per-job searches, and a tensor-core job matches the oracle."""
    sets = [make_dataset("h0", seed=101, S=420, cases=700, controls=500, k=3, top_n=10, planted=(7, 200, 411)),
            make_dataset("h1", seed=102, S=90, cases=800, controls=900, k=3, top_n=10),
            make_dataset("h2", seed=103, S=390, cases=260, controls=1100, k=3, top_n=10)]
    phs = [permuted_phenotypes(ds.phenotype, 2, seed=110 + i) for i, ds in enumerate(sets)]
    gens = [ds.genotypes for ds in sets]
    h = fc.fc_load_batch(gens, phs)
    a = fc.fc_search_batch(h, 3, 10)
    kinds = [fc.fc_batch_job_kind(h, j) for j in range(6)]
    assert kinds[0] == kinds[1] == kinds[4] == kinds[5] == 8
    assert kinds[2] == kinds[3] not in (6, 8)
    b = fc.fc_search_batch(h, 3, 10)   # replay: same lists
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    for j in (0, 3, 5):
        idx, s = fc.fc_search_job(h, j, 3, 10)
        assert np.array_equal(idx, a[0][j, :len(s)])
        np.testing.assert_allclose(s, a[1][j, :len(s)], rtol=1e-12)
    monkeypatch.setenv("FC_BATCH_TC", "0")
    h2 = fc.fc_load_batch(gens, phs)
    c = fc.fc_search_batch(h2, 3, 10)
    assert all(fc.fc_batch_job_kind(h2, j) not in (6, 8) for j in range(6))
    assert np.array_equal(a[0], c[0]) and np.array_equal(a[2], c[2])
    np.testing.assert_allclose(a[1], c[1], rtol=1e-12)
    assert tuple(a[0][0, 0]) == (7, 200, 411)
    o_idx, o_s, _ = oracle.search(gens[2], phs[2][1], 3, 10)

    def score_of(cmb):
        return float(oracle.mi(oracle.tables(gens[2], phs[2][1], 3, [cmb]), 3)[0])
    assert_topn_equal(a[0][5], a[1][5], o_idx, o_s, score_of)


def _tc3_sets(R=3):
    """Data sets for the batched tensor-core form: S >= 384 takes the tensor
    cores; t0 has both classes below 4096 (one accumulator), t1 4200 cases
    (two accumulators over the samples), t2 is small (persistent sweep).
    Replicate 0 of each is a shuffled phenotype, so that the first
    replicate's sample order is not the input order, and the last replicate
    of t0 has another case count than the others."""
    sets = [make_dataset("t0", seed=121, S=400, cases=700, controls=650, k=3, top_n=10, planted=(5, 180, 390)),
            make_dataset("t1", seed=122, S=386, cases=4200, controls=300, k=3, top_n=10, planted=(11, 90, 301)),
            make_dataset("t2", seed=123, S=60, cases=300, controls=320, k=3, top_n=10)]
    rng = np.random.default_rng(140)
    phs = []
    for i, ds in enumerate(sets):
        base = ds.phenotype[rng.permutation(ds.M)]
        ph = permuted_phenotypes(base, R, seed=130 + i)
        if i == 0:
            ph[R - 1] = (rng.random(ds.M) < 0.6).astype(np.uint8)
        phs.append(ph)
    return sets, phs


def test_batch_tc3_forms_match_sweep_and_per_job(fc, monkeypatch):
    """Both batched tensor-core forms give the lists of the all-sweep batch
    (every count exact, the same FP64 rescoring) and of per-job searches."""
    sets, phs = _tc3_sets()
    gens = [ds.genotypes for ds in sets]
    h = fc.fc_load_batch(gens, phs)
    a = fc.fc_search_batch(h, 3, 10)
    kinds = [fc.fc_batch_job_kind(h, j) for j in range(9)]
    assert kinds[:6] == [8] * 6, kinds
    assert all(x not in (6, 8) for x in kinds[6:]), kinds
    b = fc.fc_search_batch(h, 3, 10)   # replay
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    for j in (0, 2, 3, 5):
        idx, s = fc.fc_search_job(h, j, 3, 10)
        assert np.array_equal(idx, a[0][j, :len(s)])
        np.testing.assert_allclose(s, a[1][j, :len(s)], rtol=1e-12)
    monkeypatch.setenv("FC_BATCH_TC", "0")
    h2 = fc.fc_load_batch(gens, phs)
    c = fc.fc_search_batch(h2, 3, 10)
    assert np.array_equal(a[0], c[0]) and np.array_equal(a[2], c[2])
    np.testing.assert_allclose(a[1], c[1], rtol=1e-12)
    fc.fc_free(h)
    fc.fc_free(h2)


def test_batch_tc3_small_slab_buffer_and_long_lists(fc, monkeypatch):
    """A slab buffer that holds one data set's slab at a time (one launch per
    data set, slabs rebuilt in the graph) and lists long enough for the
    two-level merge give the lists of the per-job tensor-core searches."""
    sets, phs = _tc3_sets(R=2)
    gens = [ds.genotypes for ds in sets]
    monkeypatch.setenv("FC_BATCH_SLAB_MB", "1")
    h = fc.fc_load_batch(gens, phs)
    a = fc.fc_search_batch(h, 3, 200)
    assert [fc.fc_batch_job_kind(h, j) for j in range(4)] == [8] * 4
    b = fc.fc_search_batch(h, 3, 200)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    monkeypatch.setenv("FC_BATCH_TC3", "0")
    h2 = fc.fc_load_batch(gens, phs)
    c = fc.fc_search_batch(h2, 3, 200)
    assert [fc.fc_batch_job_kind(h2, j) for j in range(4)] == [6] * 4
    assert np.array_equal(a[0], c[0]) and np.array_equal(a[2], c[2])
    np.testing.assert_allclose(a[1], c[1], rtol=1e-12)
    fc.fc_free(h)
    fc.fc_free(h2)


def test_batch_tc3_one_job_against_oracle(fc):
    """One batched tensor-core job (a shuffled replicate) against the oracle."""
    ds = make_dataset("t3", seed=124, S=384, cases=300, controls=340, k=3, top_n=10, planted=(3, 150, 383))
    small = make_dataset("t4", seed=125, S=40, cases=200, controls=220, k=3, top_n=10)
    ph = permuted_phenotypes(ds.phenotype, 2, seed=150)
    ph_small = permuted_phenotypes(small.phenotype, 2, seed=151)
    h = fc.fc_load_batch([ds.genotypes, small.genotypes], [ph, ph_small])
    idx, score, cnt = fc.fc_search_batch(h, 3, 10)
    assert fc.fc_batch_job_kind(h, 1) == 8
    assert tuple(idx[0, 0]) == (3, 150, 383)
    o_idx, o_s, _ = oracle.search(ds.genotypes, ph[1], 3, 10)

    def score_of(c):
        return float(oracle.mi(oracle.tables(ds.genotypes, ph[1], 3, [c]), 3)[0])
    assert_topn_equal(idx[1, :cnt[1]], score[1, :cnt[1]], o_idx, o_s, score_of)
    fc.fc_free(h)


def test_batch_tc3_several_table_sizes(fc, monkeypatch):
    """One-accumulator data sets with 1,200, 3,000 and 6,000 samples: three
    launches of the same kernel with x ln x tables of different sizes (the
    largest with the short candidate buffer) in one graph."""
    sets = [make_dataset("s0", seed=161, S=384, cases=600, controls=600, k=3, top_n=10),
            make_dataset("s1", seed=162, S=390, cases=1400, controls=1600, k=3, top_n=10),
            make_dataset("s2", seed=163, S=386, cases=3000, controls=3000, k=3, top_n=10)]
    phs = [permuted_phenotypes(ds.phenotype, 2, seed=170 + i) for i, ds in enumerate(sets)]
    gens = [ds.genotypes for ds in sets]
    h = fc.fc_load_batch(gens, phs)
    a = fc.fc_search_batch(h, 3, 10)
    assert [fc.fc_batch_job_kind(h, j) for j in range(6)] == [8] * 6
    monkeypatch.setenv("FC_BATCH_TC3", "0")
    h2 = fc.fc_load_batch(gens, phs)
    c = fc.fc_search_batch(h2, 3, 10)
    assert [fc.fc_batch_job_kind(h2, j) for j in range(6)] == [6] * 6
    assert np.array_equal(a[0], c[0]) and np.array_equal(a[2], c[2])
    np.testing.assert_allclose(a[1], c[1], rtol=1e-12)
    fc.fc_free(h)
    fc.fc_free(h2)
