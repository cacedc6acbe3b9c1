"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and the benchmark.

This module holds workload descriptions and random-number draws only -- none of the method's
arithmetic -- so that the oracle and the CUDA path can be fed identical bytes without sharing code.
"""
from .synthetic import (CONFIG1, CONFIG2, CONFIG3, CONFIG4, config3_tensors, config4_points,
                        random_site_tensors, gaussian_complex)

__all__ = ["CONFIG1", "CONFIG2", "CONFIG3", "CONFIG4", "config3_tensors", "config4_points",
           "random_site_tensors", "gaussian_complex"]
