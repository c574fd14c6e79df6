"""B300-native BU-MBAR hot path: binning, fused log-sum-exp passes and the
Newton Hessian behind a C-ABI library (``libbumbar.so``).

``paper_2609_03541_b300.mbar`` is the ctypes binding of that library;
``paper_2609_03541_b300.workloads`` draws seeded synthetic problems.
Importing the package itself loads nothing.
"""
__all__ = ["mbar", "workloads"]
