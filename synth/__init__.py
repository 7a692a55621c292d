"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws random numbers and lays them out. It holds none of the
method's arithmetic: no Hamiltonian matrix elements, no wavefunction values, no
pencil products. Both the CUDA path and the oracle take what it produces as
plain inputs.

Workload shapes follow the paper's molecular benchmarks (Table 1: orbital,
electron and configuration counts) with synthetic integrals, because the
paper's STO-3G integrals are not available.
"""
from .generators import (  # noqa: F401
    Workload,
    WORKLOADS,
    integrals,
    rbm_theta,
    n_params,
    proxy_mc_samples,
    batched_instances,
    poisson_arrivals,
)
