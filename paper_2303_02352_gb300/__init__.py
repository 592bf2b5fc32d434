"""GB300-native aggregation-based AMG-preconditioned flexible CG (arXiv:2303.02352).

The compute path is the C-ABI CUDA library ``libamg.so`` (sources in ``csrc/``);
``amg`` is its thin Python binding.  Importing this package loads nothing:
``workloads`` (seeded inputs) is usable without a GPU.
"""
__all__ = ["amg", "workloads"]
