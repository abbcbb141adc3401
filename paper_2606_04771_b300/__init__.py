"""B300-native two-site TDVP engine for the open Fermi-Hubbard chain.

The compute path is the CUDA library ``libtdvp.so`` (sources in ``csrc/``,
C ABI in ``include/tdvp.h``); this package only marshals arguments to it.
"""
from ._lib import BondProblem, Chain, TdvpError, launch_count, lib, svd  # noqa: F401
