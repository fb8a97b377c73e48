"""B300-native optimal Lipschitz interpolation (sm_103a CUDA kernels behind a C ABI).

``paper_2606_04670_b300.lipfit`` holds the Python binding of ``liblipfit.so``;
``paper_2606_04670_b300.workloads`` holds the seeded synthetic workloads.
Importing the package itself loads nothing native; the binding raises if the
compiled library is missing (there is no CPU fallback).
"""
__all__ = ["lipfit", "workloads"]
