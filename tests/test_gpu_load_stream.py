"""Streamed loading: host genotypes copied in chunks of SNP rows that are
packed while the next chunk is copied.  The packed table must not depend on
the chunking: every pair's table from a many-chunk load equals the one-chunk
load's and the oracle's."""
import math

import numpy as np
import pytest

import oracle
from synth import make_dataset
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


@pytest.mark.parametrize("S,cases,controls,seed", [(1000, 1400, 1601, 1), (2100, 700, 800, 2), (350, 2000, 1049, 3)])
def test_chunked_load_equals_one_chunk(fc, monkeypatch, S, cases, controls, seed):
    # 1 MB chunks: 349 SNPs of 3 001 samples (3 chunks; the third reuses the
    # first staging buffer after its pack), 699 of 1 500 (4 chunks, a ragged
    # last chunk of 3 SNPs), 343 of 3 049 (2 chunks, 7 SNPs in the second).
    ds = make_dataset("ls", seed=1200 + seed, S=S, cases=cases, controls=controls, k=2, top_n=20,
                      planted=(5, S - 7))
    whole = fc.fc_load(ds.genotypes, ds.phenotype)
    monkeypatch.setenv("FC_LOAD_CHUNK_MB", "1")
    streamed = fc.fc_load(ds.genotypes, ds.phenotype)
    n = math.comb(S, 2)
    a = fc.fc_sweep_tables(whole, 2, 0, n)
    b = fc.fc_sweep_tables(streamed, 2, 0, n)
    assert np.array_equal(a, b)
    rng = np.random.default_rng(seed)
    combos = np.sort(np.stack([rng.choice(S, 3, replace=False) for _ in range(300)]), axis=1).astype(np.uint32)
    combos[0] = (0, S // 2, S - 1)
    assert np.array_equal(fc.fc_tables(streamed, 3, combos),
                          oracle.tables(ds.genotypes, ds.phenotype, 3, combos))
    g_idx, g_s = fc.fc_search(streamed, 2, 20)
    o_idx, o_s, _ = oracle.search(ds.genotypes, ds.phenotype, 2, 20)

    def score_of(c):
        return float(oracle.mi(oracle.tables(ds.genotypes, ds.phenotype, 2, [c]), 2)[0])
    assert_topn_equal(g_idx, g_s, o_idx, o_s, score_of)


@pytest.mark.parametrize("bad_snp", [0, 400, 1099])
def test_chunked_load_rejects_bad_genotype_in_any_chunk(fc, monkeypatch, bad_snp):
    monkeypatch.setenv("FC_LOAD_CHUNK_MB", "1")
    ds = make_dataset("lsbad", seed=1300, S=1100, cases=1500, controls=1500, k=2, top_n=5)
    G = ds.genotypes.copy()
    G[bad_snp, 17] = 7
    with pytest.raises(fc.FiunchoError) as e:
        fc.fc_load(G, ds.phenotype)
    assert e.value.status == fc.FC_EINVAL
    h = fc.fc_load(ds.genotypes, ds.phenotype)    # the library keeps working
    assert fc.fc_search(h, 2, 5)[0].shape == (5, 2)
