"""GB300-native multigrid-reduction (MGR) preconditioned FGMRES.

The solver lives in a C-ABI shared library (``include/mgr_gb300.h``) built
from ``csrc/``; :mod:`paper_2101_11649_gb300.mgr` is the ctypes binding.
Importing this package does not load the library.
"""
__version__ = "0.1.0"
