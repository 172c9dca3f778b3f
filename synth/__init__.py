"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This package only builds matrices and vectors (CSR arrays in host memory).  It
holds none of the inspector's or the executors' arithmetic, so both the CUDA
path and the CPU oracle can be fed from it without sharing any method code.
"""
from .matrices import (  # noqa: F401
    CSR,
    SEED_BASE,
    laplacian_5pt,
    laplacian_7pt,
    stencil_27pt,
    elasticity_blocks,
    powerlaw,
    lower_triangle,
    random_pattern,
    uniform_vector,
    workload,
    WORKLOADS,
    batch,
    batch_member,
    chain,
    banded,
)
