"""Integrity of the stored full-size oracle lists (tests/golden/topn_*.json)
on the CPU: they describe the workloads the generator makes today, their
entries are the oracle's own scores of their own tables, they are ordered
as the search orders, and the smallest one is reproduced by a fresh oracle
run.  The GPU comparison against them is in test_gpu_golden.py."""
import importlib.util
import json
import math
import os

import numpy as np
import pytest

import oracle
from synth import CONFIGS, make_batch, make_config

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
NAMES = ["C1", "C2", "C3", "C4", "P5", "P6"]


def _golden(name):
    with open(os.path.join(GOLDEN, f"topn_{name}.json")) as f:
        return json.load(f)


def _check_order(idx, score):
    for a in range(1, len(score)):
        assert score[a] <= score[a - 1]
        if score[a] == score[a - 1]:
            assert tuple(idx[a - 1]) < tuple(idx[a])


@pytest.mark.parametrize("name", NAMES)
def test_golden_describes_the_workload(name):
    g = _golden(name)
    cfg = CONFIGS[name]
    gen = g["generator"]
    assert gen["seed"] == cfg["seed"] and gen["S"] == cfg["S"]
    assert gen["cases"] == cfg["cases"] and gen["controls"] == cfg["controls"]
    assert tuple(gen["planted"]) == tuple(cfg["planted"])
    assert g["k"] == cfg["k"] and g["top_n"] == cfg["top_n"]
    assert g["tested"] == math.comb(cfg["S"], cfg["k"])
    assert len(g["idx"]) == len(g["score"]) == cfg["top_n"]
    assert tuple(g["idx"][0]) == tuple(cfg["planted"])
    _check_order(g["idx"], g["score"])


@pytest.mark.parametrize("name", NAMES)
def test_golden_scores_are_the_oracle_scores_of_their_tables(name):
    g = _golden(name)
    ds = make_config(name)
    n = len(g["idx"])
    pick = sorted(set([0, 1, 2, n // 2, n - 2, n - 1]))
    combos = np.array([g["idx"][x] for x in pick], dtype=np.uint32)
    s = oracle.mi(oracle.tables(ds.genotypes, ds.phenotype, ds.k, combos), ds.k)
    assert [float(v) for v in s] == [g["score"][x] for x in pick]


def test_golden_c1_is_reproduced_by_the_oracle():
    g = _golden("C1")
    ds = make_config("C1")
    idx, score, tested = oracle.search(ds.genotypes, ds.phenotype, ds.k, ds.top_n)
    assert tested == g["tested"]
    assert idx.astype(int).tolist() == g["idx"]
    assert [float(x) for x in score] == g["score"]


def test_golden_batched_subset_follows_its_rule():
    g = _golden("C5S")
    spec = importlib.util.spec_from_file_location("make_goldens", os.path.join(GOLDEN, "make_goldens.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    batch = make_batch()
    jobs = mg.c5_subset(batch)
    assert [(j["dataset"], j["replicate"]) for j in g["jobs"]] == [tuple(x) for x in jobs]
    for job in g["jobs"]:
        ds, ph = batch[job["dataset"]]
        assert (ds.S, ds.M, ds.cases) == (job["S"], job["M"], job["cases"])
        assert len(job["idx"]) == min(g["top_n"], math.comb(ds.S, 3))
        _check_order(job["idx"], job["score"])
    # One job's best entry, rescored by the oracle from its table.
    job = g["jobs"][0]
    ds, ph = batch[job["dataset"]]
    t = oracle.tables(ds.genotypes, ph[job["replicate"]], 3, [job["idx"][0]])
    assert float(oracle.mi(t, 3)[0]) == job["score"][0]
