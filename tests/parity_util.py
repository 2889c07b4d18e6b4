"""Comparison helpers for GPU-vs-oracle parity tests."""
import numpy as np

SCORE_REL = 1e-6      # returned (FP64-rescored) scores vs the FP64 oracle
TIE_REL = 1e-12       # scores this close are treated as ties (last-bit noise)


def _tie(a: float, b: float) -> bool:
    return abs(a - b) <= TIE_REL * max(abs(a), abs(b), 1e-300)


def assert_topn_equal(g_idx, g_score, o_idx, o_score, oracle_score_of=None):
    """Top-N lists must agree exactly on index tuples, except where scores
    tie (equal up to last-bit rounding): inside a tie group any order is
    valid, and a tie group cut by the N boundary may hold any of its
    members.  ``oracle_score_of(tuple) -> float`` checks such members."""
    g_idx = np.asarray(g_idx).reshape(len(g_score), -1)
    o_idx = np.asarray(o_idx).reshape(len(o_score), -1)
    assert len(g_score) == len(o_score), (len(g_score), len(o_score))
    n = len(o_score)
    np.testing.assert_allclose(g_score, o_score, rtol=SCORE_REL, atol=1e-12)
    i = 0
    while i < n:
        j = i + 1
        while j < n and _tie(o_score[j], o_score[i]):
            j += 1
        og = {tuple(int(x) for x in r) for r in o_idx[i:j]}
        gg = {tuple(int(x) for x in r) for r in g_idx[i:j]}
        if j < n or og == gg:
            assert og == gg, f"positions {i}..{j - 1}: oracle {sorted(og)} gpu {sorted(gg)}"
        else:
            # Last group, cut by the boundary: GPU members must be ties too.
            assert oracle_score_of is not None, f"boundary tie group differs: {og} vs {gg}"
            for c in gg - og:
                assert _tie(oracle_score_of(c), o_score[i]), c
        i = j
    # Within the GPU list, bit-equal scores are ordered by index tuple.
    for a in range(1, n):
        if g_score[a] == g_score[a - 1]:
            assert tuple(g_idx[a - 1]) < tuple(g_idx[a])
