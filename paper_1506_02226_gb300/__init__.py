"""GB300-native exact DBSCAN (the three data-parallel steps of Wang et al.,
"Design and optimization of DBSCAN Algorithm based on CUDA").

The clustering runs in libdbscan_gb300.so (hand-written sm_103a CUDA kernels
behind the C ABI in include/dbscan.h).  ``binding`` wraps that ABI with ctypes;
``api`` adds a small torch-tensor front end; ``inputs`` holds the seeded
synthetic workloads.  Nothing here computes on the CPU.
"""
from . import binding  # noqa: F401

__all__ = ["binding", "api", "inputs", "build"]
