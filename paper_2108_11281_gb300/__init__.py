"""GB300-native multilevel Monte-Carlo trace estimator (arXiv 2108.11281).

The compute path is libmlmc.so (hand-written CUDA for sm_103a, C ABI in
include/mlmc.h); ``paper_2108_11281_gb300.mlmc`` is its ctypes binding and
``workloads`` the seeded input generator.
"""
