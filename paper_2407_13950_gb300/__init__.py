"""GB300-native multiple-shooting quantum optimal control: one objective + gradient evaluation.

The compute path is the CUDA library ``libmsqoc.so`` (built from ``csrc/``) behind the C ABI
declared in ``include/msqoc.h``; ``paper_2407_13950_gb300.msqoc`` is its thin ctypes binding.
Importing this package does not load the library; ``synthetic`` (seeded workloads) is
importable without a GPU.
"""
__all__ = ["synthetic"]
