"""GB300-native lattice Boltzmann for inhomogeneous hard-sphere fluids.

``lbif`` holds the ctypes binding of the C ABI (``include/lbif.h``) whose CUDA
kernels implement the per-time-step hot path; ``inputs`` holds the seeded
workload generators; ``build`` compiles the library. Importing the package has
no side effects: the CUDA library is loaded on first use.
"""
__all__ = ["lbif", "inputs", "build"]
