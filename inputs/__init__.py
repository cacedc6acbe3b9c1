"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and the benchmark.

This module holds workload descriptions and random-number draws only -- none of the method's
arithmetic -- so that the oracle and the CUDA path can be fed identical bytes without sharing code.
"""
from .synthetic import (QUENCH_D2, QUENCH_D3, QUENCH_DA3, RANDOM_CTMRG, DISORDER_SWEEP, ED, random_ctmrg_tensors,
                        disorder_sweep_points, random_site_tensors, gaussian_complex, ed_fields)

__all__ = ["QUENCH_D2", "QUENCH_D3", "QUENCH_DA3", "RANDOM_CTMRG", "DISORDER_SWEEP", "ED", "random_ctmrg_tensors",
           "disorder_sweep_points", "random_site_tensors", "gaussian_complex", "ed_fields"]
