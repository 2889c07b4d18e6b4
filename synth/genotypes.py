"""Synthetic genotype/phenotype generator for the exhaustive epistasis search.

Every draw goes through ``numpy.random.Generator(PCG64).random()`` (uniform
doubles), whose stream numpy keeps stable across releases, so the same seed
gives the same data on every machine.  Binomial genotypes, Bernoulli
affection and permutations are built from those uniforms here rather than
through numpy's distribution methods.

Recipe (the paper's workloads are unnamed 2048-sample case/control data, so
these synthetic sets stand in for them):

* Genotypes follow Hardy-Weinberg equilibrium: SNP ``s`` has minor-allele
  frequency ``p_s`` ~ U[maf_lo, maf_hi]; genotype value ``g`` is the minor
  allele count with probabilities ``(q^2, 2pq, p^2)``, ``q = 1 - p``.
* A planted ``k``-SNP interaction has no marginal effect at any lower order.
  Each planted SNP gets the contrast ``c(g) = (P1, -(P0+P2), P1) / sd``,
  which has zero mean under its genotype distribution ``(P0, P1, P2)``; the
  penetrance is ``f = K + delta * prod_t c_t(g_t)`` with ``K`` the
  prevalence and ``delta = sqrt(h2 K (1-K))``.  Marginalising any proper
  subset of the planted SNPs leaves ``f = K``.  If ``f`` leaves [0, 1] the
  amplitude ``delta`` is halved until it fits.
* Cases and controls are filled retrospectively: individuals are drawn, the
  affection is a Bernoulli(``f``) draw, and they are kept until ``M1`` cases
  and ``M0`` controls are collected.  The sample order is then shuffled so
  cases and controls interleave.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Dataset",
    "CONFIGS",
    "make_config",
    "make_dataset",
    "make_batch",
    "random_small",
    "permuted_phenotypes",
]


@dataclass
class Dataset:
    """One case/control data set.

    ``genotypes`` is ``uint8[S][M]`` (SNP-major, values 0/1/2) and
    ``phenotype`` is ``uint8[M]`` (1 = case, 0 = control).
    """

    name: str
    genotypes: np.ndarray
    phenotype: np.ndarray
    k: int
    top_n: int
    planted: tuple = ()
    delta: float = 0.0
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def S(self) -> int:
        return int(self.genotypes.shape[0])

    @property
    def M(self) -> int:
        return int(self.genotypes.shape[1])

    @property
    def cases(self) -> int:
        return int(self.phenotype.sum())

    @property
    def controls(self) -> int:
        return self.M - self.cases


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _uniform_int(rng: np.random.Generator, lo: int, hi: int) -> int:
    """Integer uniform on [lo, hi] from one uniform double."""
    return lo + min(int(rng.random() * (hi - lo + 1)), hi - lo)


def _permutation(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random permutation of range(n) (argsort of uniform keys)."""
    return np.argsort(rng.random(n), kind="stable")


def _hwe_thresholds(maf: np.ndarray):
    q = 1.0 - maf
    t0 = q * q
    t1 = t0 + 2.0 * maf * q
    return t0, t1


def _hwe_rows(rng: np.random.Generator, maf: np.ndarray, M: int,
              out: np.ndarray, chunk_rows: int = 2048) -> None:
    """Fill ``out[S][M]`` with HWE genotypes, in row chunks to bound memory."""
    S = maf.shape[0]
    t0, t1 = _hwe_thresholds(maf)
    for r0 in range(0, S, chunk_rows):
        r1 = min(S, r0 + chunk_rows)
        u = rng.random((r1 - r0, M))
        g = (u >= t0[r0:r1, None]).astype(np.uint8)
        g += (u >= t1[r0:r1, None]).astype(np.uint8)
        out[r0:r1] = g


def _contrast(maf: float) -> np.ndarray:
    """Zero-mean, unit-variance contrast (P1, -(P0+P2), P1)/sd for one SNP."""
    q = 1.0 - maf
    P = np.array([q * q, 2.0 * maf * q, maf * maf])
    c = np.array([P[1], -(P[0] + P[2]), P[1]])
    sd = math.sqrt(float((P * c * c).sum()))
    return c / sd


def make_dataset(name: str, seed: int, S: int, cases: int, controls: int,
                 k: int, top_n: int, planted=(), maf_range=(0.05, 0.5),
                 planted_maf: float = 0.5, h2: float = 0.1,
                 prevalence: float = 0.2) -> Dataset:
    """Draw one data set following the recipe in the module docstring."""
    rng = _rng(seed)
    M = cases + controls
    planted = tuple(int(p) for p in planted)
    maf = maf_range[0] + (maf_range[1] - maf_range[0]) * rng.random(S)
    for p in planted:
        maf[p] = planted_maf
    G = np.empty((S, M), dtype=np.uint8)
    _hwe_rows(rng, maf, M, G)

    delta = 0.0
    if planted:
        K = prevalence
        delta = math.sqrt(h2 * K * (1.0 - K))
        contrasts = [_contrast(maf[p]) for p in planted]
        # Worst-case product of contrasts bounds f; halve delta until f fits.
        extreme = 1.0
        for c in contrasts:
            extreme *= float(np.abs(c).max())
        while K + delta * extreme > 1.0 or K - delta * extreme < 0.0:
            delta *= 0.5
        t = [_hwe_thresholds(np.array([maf[p]])) for p in planted]
        got_case, got_ctrl = [], []
        n_case = n_ctrl = 0
        batch = max(4096, 4 * M)
        while n_case < cases or n_ctrl < controls:
            gp = np.empty((len(planted), batch), dtype=np.uint8)
            prod = np.ones(batch)
            for i, (t0, t1) in enumerate(t):
                u = rng.random(batch)
                g = (u >= t0[0]).astype(np.uint8) + (u >= t1[0]).astype(np.uint8)
                gp[i] = g
                prod *= contrasts[i][g]
            f = K + delta * prod
            aff = rng.random(batch) < f
            ca = gp[:, aff][:, : cases - n_case]
            co = gp[:, ~aff][:, : controls - n_ctrl]
            got_case.append(ca)
            got_ctrl.append(co)
            n_case += ca.shape[1]
            n_ctrl += co.shape[1]
        gp_all = np.concatenate(got_case + got_ctrl, axis=1)
        for i, p in enumerate(planted):
            G[p] = gp_all[i]
    phen = np.concatenate([np.ones(cases, np.uint8), np.zeros(controls, np.uint8)])
    order = _permutation(rng, M)
    G = np.ascontiguousarray(G[:, order])
    phen = np.ascontiguousarray(phen[order])
    return Dataset(name=name, genotypes=G, phenotype=phen, k=k, top_n=top_n,
                   planted=planted, delta=delta, seed=seed)


def permuted_phenotypes(phenotype: np.ndarray, replicates: int, seed: int) -> np.ndarray:
    """``uint8[R][M]`` phenotype replicates: row 0 is the input, rows 1.. are
    uniform random permutations of it (case and control counts preserved)."""
    rng = _rng(seed)
    M = phenotype.shape[0]
    out = np.empty((replicates, M), dtype=np.uint8)
    out[0] = phenotype
    for r in range(1, replicates):
        out[r] = phenotype[_permutation(rng, M)]
    return out


def random_small(seed: int, S: int, M: int, cases: int | None = None) -> Dataset:
    """Tiny uniform data (genotypes uniform on {0,1,2}) for brute-force checks."""
    rng = _rng(seed)
    G = np.minimum((rng.random((S, M)) * 3).astype(np.uint8), 2)
    if cases is None:
        cases = max(1, min(M - 1, M // 2))
    phen = np.zeros(M, np.uint8)
    phen[_permutation(rng, M)[:cases]] = 1
    return Dataset(name=f"small-{seed}", genotypes=np.ascontiguousarray(G),
                   phenotype=phen, k=2, top_n=5, seed=seed)


# The five workloads.  Seeds and planted indices other than C1's are choices
# of this project (C1's come with the workload definition).
CONFIGS = {
    "C1": dict(seed=1, S=100, cases=800, controls=800, k=2, top_n=10,
               planted=(17, 63), maf_range=(0.05, 0.5)),
    "C2": dict(seed=2, S=1000, cases=2000, controls=2000, k=3, top_n=100,
               planted=(101, 502, 877), maf_range=(0.05, 0.5)),
    "C3": dict(seed=3, S=40000, cases=4096, controls=4096, k=2, top_n=1000,
               planted=(12345, 33333), maf_range=(0.01, 0.5)),
    "C4": dict(seed=4, S=300, cases=3000, controls=3000, k=4, top_n=100,
               planted=(7, 150, 222, 291), maf_range=(0.05, 0.5)),
    # Orders 5 and 6 at the SNP counts and 2048 samples of the paper's
    # single-core measurements (Table 3), with a planted interaction.
    "P5": dict(seed=6, S=152, cases=1024, controls=1024, k=5, top_n=100,
               planted=(3, 40, 77, 110, 150), maf_range=(0.05, 0.5)),
    "P6": dict(seed=7, S=76, cases=1024, controls=1024, k=6, top_n=100,
               planted=(1, 14, 30, 45, 60, 75), maf_range=(0.05, 0.5)),
    # A parity case for the order-4 tensor-core plan beyond a few hundred
    # SNPs (a mid-size version of the paper's order-4 runs, Table 4), small
    # enough in samples for an exhaustive oracle run.
    "Q4": dict(seed=8, S=600, cases=256, controls=256, k=4, top_n=100,
               planted=(9, 201, 402, 587), maf_range=(0.05, 0.5)),
    # Order 4 at the size of the paper's single-node order-4 run (Table 4:
    # 2,409 variants, 2,048 samples).
    "T4": dict(seed=9, S=2409, cases=1024, controls=1024, k=4, top_n=100,
               planted=(100, 900, 1700, 2300), maf_range=(0.05, 0.5)),
    # Orders 5 and 6 at the sizes of the paper's single-node runs (Table 4:
    # 561 and 223 variants, 2,048 samples).
    "T5": dict(seed=10, S=561, cases=1024, controls=1024, k=5, top_n=100,
               planted=(0, 120, 250, 400, 540), maf_range=(0.05, 0.5)),
    "T6": dict(seed=11, S=223, cases=1024, controls=1024, k=6, top_n=100,
               planted=(0, 40, 80, 120, 160, 200), maf_range=(0.05, 0.5)),
}

CONFIG_TITLES = {
    "C1": "order-2 exhaustive, 100 SNPs x 1,600 samples (800/800), top 10",
    "C2": "order-3 exhaustive, 1,000 SNPs x 4,000 samples (2,000/2,000), top 100",
    "C3": "order-2 all-pairs, 40,000 SNPs x 8,192 samples (4,096/4,096), top 1,000",
    "C4": "order-4 exhaustive, 300 SNPs x 6,000 samples (3,000/3,000), top 100",
    "C5": "order-3 batched, 64 data sets x 20 permutation replicates, top 10 each",
    "P5": "order-5 exhaustive, 152 SNPs x 2,048 samples (1,024/1,024), top 100",
    "P6": "order-6 exhaustive, 76 SNPs x 2,048 samples (1,024/1,024), top 100",
    "Q4": "order-4 exhaustive, 600 SNPs x 512 samples (256/256), top 100",
    "T4": "order-4 exhaustive, 2,409 SNPs x 2,048 samples (1,024/1,024), top 100",
    "T5": "order-5 exhaustive, 561 SNPs x 2,048 samples (1,024/1,024), top 100",
    "T6": "order-6 exhaustive, 223 SNPs x 2,048 samples (1,024/1,024), top 100",
}


def make_config(name: str, scale_snps: int | None = None) -> Dataset:
    """Build one of C1..C4.  ``scale_snps`` keeps every other parameter but
    truncates the SNP count (planted SNPs beyond it are dropped) for small
    parity cases."""
    cfg = dict(CONFIGS[name])
    S = cfg.pop("S")
    if scale_snps is not None:
        S = int(scale_snps)
        cfg["planted"] = tuple(p for p in cfg["planted"] if p < S)
    return make_dataset(name, S=S, **cfg)


def make_batch(n_datasets: int = 64, replicates: int = 20, seed: int = 5,
               snp_range=(200, 1500), sample_range=(1000, 8000),
               case_frac_range=(0.3, 0.7), k: int = 3, top_n: int = 10,
               planted_k: int = 3):
    """The batched workload: ``n_datasets`` data sets of uneven size, each
    with ``replicates`` phenotype permutations (replicate 0 unpermuted).

    Returns a list of ``(Dataset, phenotypes uint8[R][M])``.  Data set ``j``
    draws its sizes and planted SNPs from seed ``seed + j``.
    """
    out = []
    for j in range(n_datasets):
        rng = _rng(10_000 + seed + j)
        S = _uniform_int(rng, *snp_range)
        M = _uniform_int(rng, *sample_range)
        frac = case_frac_range[0] + (case_frac_range[1] - case_frac_range[0]) * rng.random()
        cases = min(M - 1, max(1, int(round(M * frac))))
        planted = tuple(sorted(int(x) for x in _permutation(rng, S)[:planted_k]))
        ds = make_dataset(f"C5-{j}", seed=seed + j, S=S, cases=cases,
                          controls=M - cases, k=k, top_n=top_n, planted=planted)
        ph = permuted_phenotypes(ds.phenotype, replicates, seed=20_000 + seed + j)
        out.append((ds, ph))
    return out
