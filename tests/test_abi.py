"""CPU-side checks of the C-ABI library: it builds, loads without a GPU,
exports every entry point declared in include/*.h, and its host logic
(combination counting and ranking) is right.  No compute call is made."""
import glob
import itertools
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(fc_\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2201_03331_gb300 import build, library
    build.build()
    return library()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["fc_load", "fc_search", "fc_tables", "fc_free", "fc_set_stream", "fc_strerror"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared_functions() if getattr(lib, n, None) is None]
    assert not missing, f"not exported: {missing}"


def test_binding_names_match_the_header():
    import paper_2201_03331_gb300 as fc
    for n in _declared_functions():
        assert hasattr(fc, n), f"binding lacks {n}"


@pytest.mark.parametrize("n,k,count", [
    (464, 4, 1906472876), (152, 5, 632671880), (76, 6, 218618940),
    (184865, 2, 17087441680), (3246, 3, 5694987980), (3755572, 2, 7052158645806),
    (28576, 3, 3888727096800), (2409, 4, 1399760565126), (561, 5, 454852770372),
    (223, 6, 159602946217), (17010, 3, 820134519120),
])
def test_num_combinations_matches_paper_tables(lib, n, k, count):
    import paper_2201_03331_gb300 as fc
    assert fc.fc_num_combinations(n, k) == count


def test_num_combinations_limits(lib):
    import paper_2201_03331_gb300 as fc
    assert fc.fc_num_combinations(5, 6) == 0
    assert fc.fc_num_combinations(10, 0) == 1
    assert fc.fc_num_combinations(-1, 2) == -1
    assert fc.fc_num_combinations(10**7, 6) == -1   # beyond 2^62


@pytest.mark.parametrize("S,k", [(9, 1), (9, 2), (10, 3), (11, 4), (9, 5), (8, 6)])
def test_unrank_enumerates_lexicographically(lib, S, k):
    import paper_2201_03331_gb300 as fc
    for r, cmb in enumerate(itertools.combinations(range(S), k)):
        assert tuple(fc.fc_unrank(S, k, r)) == cmb
        assert fc.fc_rank(S, k, cmb) == r


def test_unrank_large(lib):
    import paper_2201_03331_gb300 as fc
    rng = np.random.default_rng(0)
    for S, k in [(3755572, 2), (28576, 3), (2409, 4), (40000, 2), (1000, 3)]:
        total = math.comb(S, k)
        for r in list(rng.integers(0, total, 50)) + [0, total - 1]:
            c = fc.fc_unrank(S, k, int(r))
            assert all(c[i] < c[i + 1] for i in range(k - 1)) and c[-1] < S
            assert fc.fc_rank(S, k, c) == int(r)
    assert tuple(fc.fc_unrank(3755572, 2, math.comb(3755572, 2) - 1)) == (3755570, 3755571)


def test_rank_rejects_bad_tuples(lib):
    import paper_2201_03331_gb300 as fc
    with pytest.raises(fc.FiunchoError):
        fc.fc_rank(10, 3, [1, 1, 2])
    with pytest.raises(fc.FiunchoError):
        fc.fc_rank(10, 2, [3, 10])
    with pytest.raises(fc.FiunchoError):
        fc.fc_unrank(10, 2, 45)


def test_strerror_covers_every_status(lib):
    import paper_2201_03331_gb300 as fc
    for s in [0, -1, -2, -3, -4, -5, -6]:
        assert fc.fc_strerror(s) != "unknown status"


def test_load_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2201_03331_gb300 as fc
    with pytest.raises(fc.FiunchoError) as ei:
        fc.fc_load(np.zeros((3, 10), np.uint8), np.zeros(10, np.uint8))
    assert ei.value.status == fc.FC_ENODEV


def test_log2_probe_without_gpu_or_buffers_fails_cleanly(lib):
    import ctypes
    import torch
    import paper_2201_03331_gb300 as fc
    assert lib.fc_log2_approx(None, 4, None) == fc.FC_EINVAL
    assert lib.fc_log2_approx(None, -1, None) == fc.FC_EINVAL
    assert lib.fc_log2_approx(None, 0, None) == fc.FC_OK
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    n = (ctypes.c_uint32 * 4)(1, 2, 3, 4)
    out = (ctypes.c_float * 4)()
    assert lib.fc_log2_approx(n, 4, out) in (fc.FC_ENODEV, fc.FC_ECUDA)


def test_null_arguments_are_rejected(lib):
    import ctypes
    assert lib.fc_load(None, 1, 1, None, None) == -1
    out = ctypes.c_void_p()
    assert lib.fc_load(None, 1, 1, None, ctypes.byref(out)) == -1
    assert lib.fc_search(None, 2, 10, None, None, None) == -1
    assert lib.fc_tables(None, 2, None, 0, None) == -1
    lib.fc_free(None)


@pytest.mark.parametrize("S,k", [(9, 2), (9, 3), (11, 4), (10, 5), (9, 6)])
def test_extensions_of_a_prefix_form_one_rank_range(lib, S, k):
    """The rank-range searches rest on this: the combinations that begin
    with a given tuple t (of 1 to 3 SNPs) are the contiguous ranks
    [rank(t, last+1, last+2, ...), + C(S - last - 1, k - |t|))."""
    import paper_2201_03331_gb300 as fc
    ranks = {c: r for r, c in enumerate(itertools.combinations(range(S), k))}
    for T in range(1, min(3, k - 1) + 1):
        for t in itertools.combinations(range(S), T):
            last = t[-1]
            count = math.comb(S - last - 1, k - T)
            got = sorted(r for c, r in ranks.items() if c[:T] == t)
            assert len(got) == count
            if count == 0:
                continue
            first = fc.fc_rank(S, k, list(t) + [last + 1 + q for q in range(k - T)])
            assert got == list(range(first, first + count))
