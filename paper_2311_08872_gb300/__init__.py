"""GB300-native MLMC for the 2-D Dean--Kawasaki equation (arXiv 2311.08872).

The compute path lives in ``libmlmc_dk.so`` (CUDA for sm_103a behind the C-ABI
declared in ``include/mlmc_dk.h``); ``mlmc_dk`` is the thin ctypes binding.
Importing the package does not load the library; ``workloads`` holds only the
seeded synthetic inputs.
"""
__all__ = ["workloads"]
