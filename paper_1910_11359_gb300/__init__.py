"""GB300-native iPEPS real-time evolution of 2D many-body-localised lattices (arXiv:1910.11359).

The compute path is libipeps.so (hand-written CUDA for sm_103a behind a C ABI, include/ipeps.h);
this package only loads it and marshals arguments.
"""
from ._lib import (FP64, SPLIT_BF16X3, SPLIT_TF32X3, IPEPS, IpepsError, footprint_bytes, fp64_peak_tflops,
                   launch_count, lib, profile_enable, profile_read, profile_tc_executed,
                   profile_counters, ed_max_sites, ed_run)

__all__ = ["FP64", "SPLIT_BF16X3", "SPLIT_TF32X3", "IPEPS", "IpepsError", "footprint_bytes",
           "fp64_peak_tflops", "launch_count", "lib", "profile_enable", "profile_read",
           "profile_tc_executed", "profile_counters", "ed_max_sites", "ed_run"]
