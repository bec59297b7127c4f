"""Seeded synthetic inputs shared by the oracle tests, the GPU parity tests and the benchmark.

This package only builds inputs: sparse SPD matrices in CSR form, right-hand sides and
system mixes. It contains none of the solver's arithmetic (no SpMV, preconditioner, vector
recurrences or dot products of the method), so the oracle and the CUDA path can both be fed
from it without sharing any of their own code.
"""
from .rng import mix64, u64_stream, uniform, uniform_pm1, normal
from .matrices import (
    CSR,
    poisson2d,
    poisson3d,
    varcoeff2d,
    varcoeff3d,
    rgg_laplacian,
    box125,
    box125_nnz,
    box_stencil,
    hadamard_spd,
    batch_mix,
    serving_mix,
    rhs_uniform,
    xtrue_uniform,
    build_spec,
)

__all__ = [
    "mix64", "u64_stream", "uniform", "uniform_pm1", "normal",
    "CSR", "poisson2d", "poisson3d", "varcoeff2d", "varcoeff3d", "rgg_laplacian",
    "box125", "box125_nnz", "box_stencil", "hadamard_spd", "batch_mix", "serving_mix", "rhs_uniform", "xtrue_uniform", "build_spec",
]
