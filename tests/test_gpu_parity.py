"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tables and index sets are compared exactly; FP64-rescored scores within
1e-6 relative; the FP32 sweep scores within the derived FP32 error bound.
"""
import itertools
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from synth import make_config, make_dataset, random_small
from tests.parity_util import assert_topn_equal

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def fp32_bound(k, M):
    """Bound on |FP32 sweep score - exact MI| in nats: 2 * 2^-24 *
    (2 ln M + (2*3^k + 6) ln 2).  With u = 2^-24: each ln table entry errs
    by u ln M, each difference of two by 2u ln M plus its own rounding, each
    product and each of the 2*3^k accumulations by u times a partial sum
    bounded by N ln 2, the final scaling and subtraction by 3u ln 2; divided
    by N and doubled for margin."""
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


def _oracle_score_fn(ds, k):
    def f(cmb):
        return float(oracle.mi(oracle.tables(ds.genotypes, ds.phenotype, k, [cmb]), k)[0])
    return f


# ---- tables -----------------------------------------------------------------

@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_tables_match_oracle(fc, k):
    ds = make_dataset("t", seed=100 + k, S=13, cases=150, controls=173, k=k, top_n=5)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    combos = list(itertools.combinations(range(ds.S), k))
    rng = np.random.default_rng(k)
    if len(combos) > 400:
        combos = [combos[i] for i in rng.choice(len(combos), 400, replace=False)]
    combos = np.array(combos, dtype=np.uint32)
    assert np.array_equal(fc.fc_tables(h, k, combos), oracle.tables(ds.genotypes, ds.phenotype, k, combos))
    # Any SNP order: cells follow the given order (first SNP most significant).
    rev = combos[:, ::-1].copy()
    assert np.array_equal(fc.fc_tables(h, k, rev), oracle.tables(ds.genotypes, ds.phenotype, k, rev))


@pytest.mark.parametrize("name", ["C1", "C2", "C4"])
def test_tables_match_oracle_full_size_sampled(fc, name):
    ds = make_config(name)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    assert fc.fc_info(h) == (ds.S, ds.M, ds.cases, ds.controls)
    rng = np.random.default_rng(7)
    k = ds.k
    combos = np.sort(np.stack([rng.choice(ds.S, k, replace=False) for _ in range(3000)]), axis=1)
    combos = combos.astype(np.uint32)
    combos[0] = np.arange(k)
    combos[1] = np.arange(ds.S - k, ds.S)
    got = fc.fc_tables(h, k, combos)
    assert np.array_equal(got, oracle.tables(ds.genotypes, ds.phenotype, k, combos))
    assert np.all(got[:, :, 0].sum(axis=1) == ds.cases)
    assert np.all(got[:, :, 1].sum(axis=1) == ds.controls)


# ---- FP32 sweep scores --------------------------------------------------------

@pytest.mark.parametrize("k,S,cases,controls", [(1, 40, 300, 211), (2, 45, 700, 900),
                                                (3, 30, 2000, 2000), (4, 20, 1500, 1437)])
def test_sweep_scores_within_fp32_bound(fc, k, S, cases, controls):
    ds = make_dataset("s", seed=200 + k, S=S, cases=cases, controls=controls, k=k, top_n=5)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    total = math.comb(S, k)
    s32 = fc.fc_scores(h, k, 0, total)
    combos = np.array(list(itertools.combinations(range(S), k)), dtype=np.uint32)
    s64 = oracle.mi(oracle.tables(ds.genotypes, ds.phenotype, k, combos), k)
    err = np.abs(s32.astype(np.float64) - s64)
    assert err.max() <= fp32_bound(k, ds.M), (err.max(), fp32_bound(k, ds.M))
    # A rank sub-range returns the same values.
    a = total // 3
    b = min(total, a + 57)
    assert np.array_equal(fc.fc_scores(h, k, a, b - a), s32[a:b])


def test_sweep_scores_full_size_sampled_c2(fc):
    ds = make_config("C2")
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    total = math.comb(ds.S, 3)
    rng = np.random.default_rng(3)
    for start in [0, int(rng.integers(0, total - 5000)), total - 4000]:
        n = min(4000, total - start)
        s32 = fc.fc_scores(h, 3, start, n)
        combos = np.array([fc.fc_unrank(ds.S, 3, r) for r in range(start, start + n)], dtype=np.uint32)
        s64 = oracle.mi(oracle.tables(ds.genotypes, ds.phenotype, 3, combos), 3)
        assert np.abs(s32 - s64).max() <= fp32_bound(3, ds.M)


# ---- search -----------------------------------------------------------------

SEARCH_CASES = [
    # name, dataset kwargs, k, top_n
    ("k1", dict(seed=31, S=50, cases=400, controls=350), 1, 10),
    ("k2", dict(seed=32, S=80, cases=777, controls=801, planted=(10, 70)), 2, 25),
    ("k3", dict(seed=33, S=110, cases=2000, controls=2000, planted=(5, 50, 100)), 3, 100),
    ("k4", dict(seed=34, S=34, cases=3000, controls=3000, planted=(3, 12, 20, 33)), 4, 100),
    ("k3-ragged", dict(seed=35, S=47, cases=1001, controls=333), 3, 64),
]


@pytest.mark.parametrize("case", SEARCH_CASES, ids=[c[0] for c in SEARCH_CASES])
def test_search_matches_oracle(fc, case):
    name, kw, k, top_n = case
    ds = make_dataset(name, k=k, top_n=top_n, **kw)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    g_idx, g_s = fc.fc_search(h, k, top_n)
    o_idx, o_s, tested = oracle.search(ds.genotypes, ds.phenotype, k, top_n)
    assert tested == math.comb(ds.S, k)
    assert_topn_equal(g_idx, g_s, o_idx, o_s, _oracle_score_fn(ds, k))
    if "planted" in kw:
        assert tuple(g_idx[0]) == tuple(kw["planted"])


def test_search_c1_full(fc):
    ds = make_config("C1")
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    g_idx, g_s = fc.fc_search(h, 2, ds.top_n)
    o_idx, o_s, _ = oracle.search(ds.genotypes, ds.phenotype, 2, ds.top_n)
    assert_topn_equal(g_idx, g_s, o_idx, o_s, _oracle_score_fn(ds, 2))
    assert tuple(g_idx[0]) == (17, 63)


@pytest.mark.parametrize("name", ["C2", "C4"])
def test_search_full_size_properties(fc, name):
    """Full-size search: every returned combination's exact table and FP64
    score agree with the oracle, the planted interaction ranks first, and no
    combination of a random sample scores above the cut."""
    ds = make_config(name)
    k = ds.k
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    g_idx, g_s = fc.fc_search(h, k, ds.top_n)
    assert len(g_s) == ds.top_n
    o_tab = oracle.tables(ds.genotypes, ds.phenotype, k, g_idx)
    assert np.array_equal(fc.fc_tables(h, k, g_idx), o_tab)
    np.testing.assert_allclose(g_s, oracle.mi(o_tab, k), rtol=1e-6, atol=1e-12)
    assert np.all(np.diff(g_s) <= 1e-15)
    assert tuple(g_idx[0]) == tuple(ds.planted)
    rng = np.random.default_rng(11)
    total = math.comb(ds.S, k)
    ranks = rng.integers(0, total, 20000)
    combos = np.array([fc.fc_unrank(ds.S, k, int(r)) for r in ranks], dtype=np.uint32)
    s = oracle.mi(oracle.tables(ds.genotypes, ds.phenotype, k, combos), k)
    returned = {tuple(int(x) for x in r) for r in g_idx}
    for c, v in zip(combos, s):
        if tuple(int(x) for x in c) not in returned:
            assert v <= g_s[-1] * (1 + 1e-12)


def test_search_is_deterministic(fc):
    ds = make_dataset("det", seed=41, S=90, cases=900, controls=1100, k=3, top_n=50)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    a = fc.fc_search(h, 3, 50)
    b = fc.fc_search(h, 3, 50)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


# ---- edge cases ---------------------------------------------------------------

def test_top_n_larger_than_combinations(fc):
    ds = random_small(51, S=7, M=60)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    g_idx, g_s = fc.fc_search(h, 3, 100)
    o_idx, o_s, _ = oracle.search(ds.genotypes, ds.phenotype, 3, 100)
    assert len(g_idx) == math.comb(7, 3)
    assert_topn_equal(g_idx, g_s, o_idx, o_s, _oracle_score_fn(ds, 3))


def test_top_n_zero_and_k_equals_s(fc):
    ds = random_small(52, S=4, M=33)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    idx, s = fc.fc_search(h, 2, 0)
    assert len(idx) == 0
    idx, s = fc.fc_search(h, 4, 3)
    assert idx.tolist() == [[0, 1, 2, 3]]
    assert s[0] == pytest.approx(oracle.mi(oracle.tables(ds.genotypes, ds.phenotype, 4, [[0, 1, 2, 3]]), 4)[0],
                                 rel=1e-12)


@pytest.mark.parametrize("M,cases", [(1, 1), (2, 1), (37, 1), (129, 128), (300, 0), (300, 300)])
def test_tiny_and_one_class_inputs(fc, M, cases):
    ds = random_small(53 + M, S=9, M=M, cases=cases)
    ph = np.zeros(M, np.uint8)
    ph[:cases] = 1
    h = fc.fc_load(ds.genotypes, ph)
    g_idx, g_s = fc.fc_search(h, 2, 12)
    o_idx, o_s, _ = oracle.search(ds.genotypes, ph, 2, 12)
    ds.phenotype = ph
    assert_topn_equal(g_idx, g_s, o_idx, o_s, _oracle_score_fn(ds, 2))
    combos = np.array(list(itertools.combinations(range(9), 2)), dtype=np.uint32)
    assert np.array_equal(fc.fc_tables(h, 2, combos), oracle.tables(ds.genotypes, ph, 2, combos))


def test_monomorphic_snps(fc):
    ds = make_dataset("mono", seed=61, S=40, cases=500, controls=500, k=2, top_n=10)
    G = ds.genotypes.copy()
    G[3] = 0
    G[17] = 2
    G[18] = 1
    h = fc.fc_load(G, ds.phenotype)
    g_idx, g_s = fc.fc_search(h, 2, 780)
    o_idx, o_s, _ = oracle.search(G, ds.phenotype, 2, 780)
    ds.genotypes = G
    assert_topn_equal(g_idx, g_s, o_idx, o_s, _oracle_score_fn(ds, 2))


def test_load_device_matches_host_load(fc):
    import torch
    ds = make_dataset("dev", seed=71, S=64, cases=333, controls=444, k=2, top_n=10)
    h1 = fc.fc_load(ds.genotypes, ds.phenotype)
    h2 = fc.fc_load_device(torch.from_numpy(ds.genotypes).cuda(), torch.from_numpy(ds.phenotype).cuda())
    a = fc.fc_search(h1, 2, 10)
    b = fc.fc_search(h2, 2, 10)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_caller_stream(fc):
    import torch
    ds = make_dataset("st", seed=72, S=50, cases=400, controls=400, k=2, top_n=10)
    h = fc.fc_load(ds.genotypes, ds.phenotype)
    ref = fc.fc_search(h, 2, 10)
    s = torch.cuda.Stream()
    fc.fc_set_stream(h, s)
    got = fc.fc_search(h, 2, 10)
    fc.fc_set_stream(h, None)
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])


# ---- errors -----------------------------------------------------------------

def test_invalid_inputs_are_rejected(fc):
    G = np.zeros((5, 20), np.uint8)
    ph = np.array([1, 0] * 10, np.uint8)
    bad = G.copy(); bad[2, 7] = 3
    with pytest.raises(fc.FiunchoError) as e:
        fc.fc_load(bad, ph)
    assert e.value.status == fc.FC_EINVAL
    bph = ph.copy(); bph[4] = 2
    with pytest.raises(fc.FiunchoError) as e:
        fc.fc_load(G, bph)
    assert e.value.status == fc.FC_EINVAL
    h = fc.fc_load(G, ph)
    for k in (0, 6, 7):          # k = 6 exceeds S = 5; 7 exceeds the maximum order
        with pytest.raises(fc.FiunchoError) as e:
            fc.fc_search(h, k, 3)
        assert e.value.status == fc.FC_EINVAL
    with pytest.raises(fc.FiunchoError) as e:
        fc.fc_search(h, 2, 10**6)
    assert e.value.status == fc.FC_ERANGE
    with pytest.raises(fc.FiunchoError) as e:
        fc.fc_tables(h, 2, [[0, 5]])
    assert e.value.status == fc.FC_EINVAL
    big = np.zeros((2, 70000), np.uint8)
    with pytest.raises(fc.FiunchoError) as e:
        fc.fc_load(big, np.ones(70000, np.uint8))
    assert e.value.status == fc.FC_ERANGE


def test_injected_allocation_failure_is_reported():
    """FC_FAULT_ALLOC makes the n-th device allocation fail on the host side;
    the call reports FC_ENOMEM and the process can keep using the library."""
    code = (
        "import numpy as np, paper_2201_03331_gb300 as fc\n"
        "G = np.zeros((4, 50), np.uint8); ph = np.array([1, 0] * 25, np.uint8)\n"
        "try:\n"
        "    fc.fc_load(G, ph); print('NOFAIL')\n"
        "except fc.FiunchoError as e:\n"
        "    print('STATUS', e.status)\n"
        "h = fc.fc_load(G, ph); print('OK', fc.fc_search(h, 2, 3)[0].shape)\n"
    )
    for n in (1, 3, 5):
        env = dict(os.environ, FC_FAULT_ALLOC=str(n))
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=300)
        assert r.returncode == 0, r.stderr
        assert f"STATUS {-3}" in r.stdout and "OK (3, 2)" in r.stdout, r.stdout


def test_injected_launch_failure_is_reported():
    code = (
        "import numpy as np, paper_2201_03331_gb300 as fc\n"
        "G = np.zeros((4, 50), np.uint8); ph = np.array([1, 0] * 25, np.uint8)\n"
        "try:\n"
        "    fc.fc_load(G, ph); print('NOFAIL')\n"
        "except fc.FiunchoError as e:\n"
        "    print('STATUS', e.status)\n"
    )
    env = dict(os.environ, FC_FAULT_LAUNCH="1")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    assert f"STATUS {-4}" in r.stdout, r.stdout
