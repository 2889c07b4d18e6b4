"""Full-size parity: fc_search's whole top-N list at each workload's full
size against the oracle's exhaustive search, stored in tests/golden/ by
tests/golden/make_goldens.py (which calls only oracle/ and synth/).

Index tuples must agree exactly, FP64-rescored scores within 1e-6 relative
(tie groups that the top-N boundary cuts may hold any of their members; such
members are checked against the oracle's own score).  The batched workload
is checked on the stored subset of its jobs, searched inside the full
64 x 20 batch.
"""
import json
import os

import numpy as np
import pytest

import oracle
from synth import make_batch, make_config
from tests.parity_util import assert_topn_equal

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# Path each workload takes by default (fc_last_search_kind): 3 the
# inclusion-exclusion sweep, 2 / 6 / 7 the order-2 / order-3 / orders 4-6
# tensor-core kernels.
DEFAULT_KIND = {"C1": 3, "C2": 6, "C3": 2, "C4": 7, "P5": 7, "P6": 7}


def _golden(name):
    path = os.path.join(GOLDEN, f"topn_{name}.json")
    with open(path) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def fc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2201_03331_gb300 as fcm
    from paper_2201_03331_gb300 import build
    build.build()
    return fcm


def _score_fn(G, ph, k):
    def f(c):
        return float(oracle.mi(oracle.tables(G, ph, k, [c]), k)[0])
    return f


@pytest.mark.parametrize("name", ["C1", "C2", "C3", "C4", "P5", "P6"])
def test_full_size_top_n_equals_oracle(fc, name):
    g = _golden(name)
    ds = make_config(name)
    assert (ds.S, ds.cases, ds.controls, ds.k, ds.top_n) == (
        g["generator"]["S"], g["generator"]["cases"], g["generator"]["controls"], g["k"], g["top_n"])
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    idx, s = fc.fc_search(h, ds.k, ds.top_n)
    assert fc.fc_last_search_kind(h) == DEFAULT_KIND[name]
    o_idx = np.array(g["idx"], dtype=np.uint32)
    o_s = np.array(g["score"], dtype=np.float64)
    assert_topn_equal(idx, s, o_idx, o_s, _score_fn(ds.genotypes, ds.phenotype, ds.k))
    assert tuple(int(x) for x in idx[0]) == tuple(g["generator"]["planted"])
    fc.fc_free(h)


def test_batched_subset_equals_oracle(fc):
    g = _golden("C5S")
    batch = make_batch()
    R = g["batch"]["replicates"]
    assert len(batch) == g["batch"]["n_datasets"] and batch[0][1].shape[0] == R
    h = fc.fc_load_batch([ds.genotypes for ds, _ in batch], [ph for _, ph in batch])
    idx, s, cnt = fc.fc_search_batch(h, 3, g["top_n"])
    kinds = set()
    for job in g["jobs"]:
        j, r = job["dataset"], job["replicate"]
        ds, ph = batch[j]
        assert (ds.S, ds.M) == (job["S"], job["M"])
        jj = j * R + r
        kinds.add(fc.fc_batch_job_kind(h, jj))
        n = int(cnt[jj])
        assert_topn_equal(idx[jj][:n], s[jj][:n], np.array(job["idx"], dtype=np.uint32),
                          np.array(job["score"]), _score_fn(ds.genotypes, ph[r], 3))
    # The subset holds jobs of both batched paths (persistent sweep and
    # batched tensor-core launches).
    assert 8 in kinds and len(kinds) >= 2, kinds
    fc.fc_free(h)
