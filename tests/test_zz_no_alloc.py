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
import numpy as np
import pytest

from synth import make_dataset
from tests.parity_util import SCORE_REL

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
