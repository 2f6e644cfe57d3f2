"""GB300 (sm_103a) implementation of the time step of the MRT lattice Boltzmann
scheme for the anisotropic Cahn-Hilliard equation (arXiv 2501.03759).

The compute lives in the CUDA library ``liblbch.so`` (sources in ``csrc/``,
C-ABI in ``include/lbch.h``); ``paper_2501_03759_gb300.lbch`` is its thin ctypes
binding. Importing this package loads nothing; the binding loads the library on
first use and raises if it has not been built (see ``build.build``).
"""
