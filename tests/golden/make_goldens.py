#!/usr/bin/env python3
"""Write the oracle's full-size top-N lists to ``tests/golden/topn_*.json``.

This script calls only the CPU oracle (``oracle/``) and the seeded input
generator (``synth/``): every stored index tuple and score is the oracle's
exhaustive search (Algorithm 1: every k-combination counted sample by sample,
FP64 mutual information, ordered by score descending then index tuple
ascending) on the synthetic workloads, never a value from the CUDA path.

    python tests/golden/make_goldens.py                # every workload
    python tests/golden/make_goldens.py C2 C4          # some of them
    python tests/golden/make_goldens.py --threads 7 C3

Workloads: C1 (order 2, 100 x 1,600), C2 (order 3, 1,000 x 4,000), C3
(order 2 all-pairs, 40,000 x 8,192), C4 (order 4, 300 x 6,000), P5 / P6
(orders 5 and 6 at 152 / 76 SNPs x 2,048 samples), Q4 (order 4, 600 x 512,
a parity case for the order-4 tensor-core plan), and C5S, a fixed subset
of the batched workload (64 data sets x 20 phenotype replicates, order 3,
top 10 per job) -- the whole batch is about 1.5e11 combinations, hours of
oracle time, so the subset below is stored and labelled as a subset.
"""
import argparse
import hashlib
import json
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from synth import CONFIGS, make_batch, make_config  # noqa: E402

SINGLE = ["C1", "C2", "C4", "P6", "P5", "Q4", "C3"]

# The batched-workload subset: one replicate (number j mod 20) of every data
# set j whose search costs at most C5S_MAX_WORK sample-combinations, the two
# data sets with the most SNPs among those at most C5S_BIG_WORK (the largest
# tensor-core jobs whose oracle run stays short), and all 20 replicates of the
# two data sets with the fewest SNPs.  Fixed by these rules, not by hand.
C5S_MAX_WORK = 1.2e11
C5S_BIG_WORK = 7.0e11


def c5_subset(batch):
    work = [math.comb(ds.S, 3) * ds.M for ds, _ in batch]
    R = batch[0][1].shape[0]
    jobs = set()
    for j, w in enumerate(work):
        if w <= C5S_MAX_WORK:
            jobs.add((j, j % R))
    big = sorted((j for j, w in enumerate(work) if C5S_MAX_WORK < w <= C5S_BIG_WORK),
                 key=lambda j: -batch[j][0].S)[:2]
    for j in big:
        jobs.add((j, j % R))
    for j in sorted(range(len(batch)), key=lambda j: batch[j][0].S)[:2]:
        for r in range(R):
            jobs.add((j, r))
    return sorted(jobs)


def _sha(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def _write(name, obj):
    path = os.path.join(HERE, f"topn_{name}.json")
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(obj, f, separators=(",", ":"))
        f.write("\n")
    os.replace(tmp, path)
    return path


def make_single(name, threads):
    cfg = CONFIGS[name]
    ds = make_config(name)
    t0 = time.time()
    idx, score, tested = oracle.search(ds.genotypes, ds.phenotype, ds.k, ds.top_n, threads)
    dt = time.time() - t0
    assert tested == math.comb(ds.S, ds.k)
    obj = {
        "what": f"oracle top-{ds.top_n} of the full exhaustive order-{ds.k} search",
        "workload": name,
        "generator": {"seed": cfg["seed"], "S": ds.S, "cases": ds.cases,
                      "controls": ds.controls, "planted": list(cfg["planted"]),
                      "maf_range": list(cfg["maf_range"])},
        "k": ds.k, "top_n": ds.top_n, "tested": int(tested),
        "oracle_source_sha256_16": _sha(os.path.join(ROOT, "oracle", "oracle.c")),
        "oracle_seconds": round(dt, 1), "threads": threads or os.cpu_count(),
        "idx": idx.astype(int).tolist(),
        "score": [float(x) for x in score],
    }
    return _write(name, obj), dt


def make_c5_subset(threads):
    batch = make_batch()
    jobs = c5_subset(batch)
    out = []
    t0 = time.time()
    for j, r in jobs:
        ds, ph = batch[j]
        idx, score, tested = oracle.search(ds.genotypes, ph[r], 3, ds.top_n, threads)
        assert tested == math.comb(ds.S, 3)
        out.append({"dataset": j, "replicate": r, "S": ds.S, "M": ds.M, "cases": ds.cases,
                    "idx": idx.astype(int).tolist(), "score": [float(x) for x in score]})
    dt = time.time() - t0
    obj = {
        "what": ("oracle top-10 of the order-3 search for a fixed subset of the batched "
                 "workload's (data set, replicate) jobs"),
        "workload": "C5S",
        "subset_rule": (f"replicate j mod 20 of every data set j with C(S,3)*M <= {C5S_MAX_WORK:g}; "
                        f"the two data sets with most SNPs among C(S,3)*M <= {C5S_BIG_WORK:g}; "
                        "all replicates of the two data sets with fewest SNPs"),
        "batch": {"n_datasets": len(batch), "replicates": int(batch[0][1].shape[0]), "seed": 5},
        "k": 3, "top_n": 10, "n_jobs": len(out),
        "oracle_source_sha256_16": _sha(os.path.join(ROOT, "oracle", "oracle.c")),
        "oracle_seconds": round(dt, 1), "threads": threads or os.cpu_count(),
        "jobs": out,
    }
    return _write("C5S", obj), dt


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="*", default=SINGLE + ["C5S"])
    ap.add_argument("--threads", type=int, default=0, help="oracle threads (0 = all cores)")
    a = ap.parse_args()
    for name in a.names:
        if name == "C5S":
            path, dt = make_c5_subset(a.threads)
        else:
            path, dt = make_single(name, a.threads)
        print(f"{name}: {path} ({dt:.1f} s)", flush=True)


if __name__ == "__main__":
    main()
