"""GB300-native solver for the coupled finite-difference / lattice-Boltzmann scheme for
catalytic flow (Kulyk, Berger, Smith, Harting, arXiv:1804.07588).

``fdlbm`` is the Python binding of the C-ABI CUDA library ``libfdlbm.so``;
``workloads`` describes seeded synthetic problems; ``build`` compiles the library.
Importing the package does not load CUDA code.
"""
__all__ = ["fdlbm", "workloads", "build"]
