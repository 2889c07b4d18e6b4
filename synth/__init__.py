"""Seeded synthetic case/control genotype data.

This package only draws inputs: genotypes, phenotypes, planted interactions
and phenotype permutations.  It holds none of the search arithmetic
(contingency tables, entropies, ranking), so both the CUDA path and the CPU
oracle can be fed from it without sharing any of the method's code.
"""
from .genotypes import (  # noqa: F401
    Dataset,
    CONFIGS,
    make_config,
    make_dataset,
    make_batch,
    random_small,
    permuted_phenotypes,
)
