"""GB300-native half-range Gauss-Hermite lattice Boltzmann step (arXiv:1708.03249).

The compute path is the C-ABI library ``libhlb`` (CUDA for sm_103a, built
in-tree by ``paper_1708_03249_gb300.build``); ``paper_1708_03249_gb300.hlb``
is its thin ctypes binding.  Importing this package loads nothing; the
binding loads the library on first use and raises if it is missing.
"""
