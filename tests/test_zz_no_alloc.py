"""The allocation-free search entry point, fc_search_static.

Some callers cannot call cudaMalloc while they search: cudaMalloc/cudaFree
may synchronise the device and take a driver-wide lock, and applications
whose own allocator owns the device memory budget forbid them.  For those
callers fc_search_static takes its work area from a fixed 8 MiB array in
the library's device image.  These tests call it through the C ABI and
check that it returns what fc_search returns, twice in a row (the array is
shared by every call and keeps the previous call's contents), and that a
search too large for the array is refused.

This file is collected last so that a run stopping at the first failure
has already run every other test.
"""
import os

import numpy as np
import pytest

import oracle
from synth import make_dataset
from tests.parity_util import SCORE_REL, assert_topn_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2201_03331_gb300 as fcm
    from paper_2201_03331_gb300 import build
    build.build()
    return fcm


@pytest.mark.parametrize("k,top_n", [(3, 100), (2, 25)])
def test_static_search_matches_fc_search_twice(fc, k, top_n):
    ds = make_dataset("noalloc", seed=91, S=140, cases=1200, controls=1300, k=k, top_n=top_n,
                      planted=(7, 70, 133)[:k])
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    ref_idx, ref_s = fc.fc_search(h, k, top_n)
    for _ in range(2):
        idx, s = fc.fc_search_static(h, k, top_n)
        assert np.array_equal(idx, ref_idx)
        np.testing.assert_allclose(s, ref_s, rtol=SCORE_REL, atol=1e-12)
    assert tuple(idx[0]) == (7, 70, 133)[:k]


def test_static_search_two_data_sets_in_a_row(fc):
    # The shared array keeps the previous call's contents; a different search
    # right after must not see them.
    a = make_dataset("na-a", seed=92, S=90, cases=700, controls=650, k=3, top_n=50)
    b = make_dataset("na-b", seed=93, S=75, cases=400, controls=900, k=3, top_n=20)
    ha, hb = fc.fc_load(a.genotypes, a.phenotype), fc.fc_load(b.genotypes, b.phenotype)
    ra, rb = fc.fc_search(ha, 3, 50), fc.fc_search(hb, 3, 20)
    for h, ref, n in ((ha, ra, 50), (hb, rb, 20), (ha, ra, 50)):
        idx, s = fc.fc_search_static(h, 3, n)
        assert np.array_equal(idx, ref[0])
        np.testing.assert_allclose(s, ref[1], rtol=SCORE_REL, atol=1e-12)


def test_static_search_rejects_work_beyond_the_array(fc):
    ds = make_dataset("na-big", seed=94, S=200, cases=500, controls=500, k=2, top_n=2000)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    with pytest.raises(fc.FiunchoError) as e:
        fc.fc_search_static(h, 2, 2000)
    assert e.value.status == fc.FC_ERANGE
    assert "static scratch" in str(e.value)
    # The regular entry point still serves it.
    idx, _ = fc.fc_search(h, 2, 2000)
    assert len(idx) == 2000


def test_static_search_first_on_a_fresh_handle_matches_oracle(fc):
    # No fc_search has run on this handle, so the operands fc_search builds
    # on first use (inclusion-exclusion tables) do not exist: the static
    # search takes a sweep that needs none, with the same results.
    ds = make_dataset("na-fresh", seed=95, S=120, cases=800, controls=900, k=3, top_n=40,
                      planted=(11, 60, 101))
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    idx, s = fc.fc_search_static(h, 3, 40)
    o_idx, o_s, _ = oracle.search(ds.genotypes, ds.phenotype, 3, 40)

    def score_of(c):
        return float(oracle.mi(oracle.tables(ds.genotypes, ds.phenotype, 3, [c]), 3)[0])
    assert_topn_equal(idx, s, o_idx, o_s, score_of)
    assert tuple(idx[0]) == (11, 60, 101)


def test_static_search_allocates_nothing(fc):
    """With every device allocation of the library made to fail
    (FC_FAULT_ALLOC_ALL), fc_search_static still succeeds, and the device's
    free memory is the same before and after it."""
    import torch
    ds = make_dataset("na-none", seed=96, S=110, cases=600, controls=700, k=3, top_n=30)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    ref = fc.fc_search(h, 3, 30)
    fc.fc_search_static(h, 3, 30)          # the array's module is loaded by now
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    os.environ["FC_FAULT_ALLOC_ALL"] = "1"
    try:
        # The switch is live: a fresh handle's fc_search must grow scratch.
        h2 = None
        with pytest.raises(fc.FiunchoError) as e:
            h2 = fc.fc_load(ds.genotypes, ds.phenotype)
        assert e.value.status == fc.FC_ENOMEM
        assert h2 is None
        for _ in range(2):
            idx, s = fc.fc_search_static(h, 3, 30)
            assert np.array_equal(idx, ref[0])
            np.testing.assert_allclose(s, ref[1], rtol=SCORE_REL, atol=1e-12)
    finally:
        del os.environ["FC_FAULT_ALLOC_ALL"]
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_static_search_with_right_chunks_allocates_nothing(fc, monkeypatch):
    """Orders 4-6 with the right tuple rows in chunks: once fc_search has
    built the operands, the static search rebuilds each chunk's rows into
    the kept buffer without allocating (every device allocation made to
    fail), with fc_search's results."""
    monkeypatch.setenv("FC_QUADS_PATH", "tc")
    monkeypatch.setenv("FC_TUPLES_SLAB_MB", "6")
    ds = make_dataset("na-chunks", seed=97, S=30, cases=300, controls=290, k=5, top_n=20,
                      planted=(2, 8, 13, 20, 27))
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    ref = fc.fc_search(h, 5, 20)
    assert fc.fc_last_search_kind(h) == 7
    monkeypatch.setenv("FC_FAULT_ALLOC_ALL", "1")
    for _ in range(2):
        idx, s = fc.fc_search_static(h, 5, 20)
        assert fc.fc_last_search_kind(h) == 7
        assert np.array_equal(idx, ref[0])
        np.testing.assert_allclose(s, ref[1], rtol=SCORE_REL, atol=1e-12)
