"""GB300-native fourth-order cut-cell elliptic solver (arxiv 2504.00724).

Thin Python binding over the C ABI in include/ccm.h (libccm.so, built in-tree by
``build.py``).  The binding only marshals arguments: setup, operator application and the
multigrid solve run in the library's host C++ and sm_103a CUDA kernels.  Importing the
package loads the library and raises if it is missing; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

from .binding import (CCM_DIRICHLET, CCM_FP64, CCM_MIXED, CCM_NEUMANN, CCM_NONE, CCM_ROBIN, CcmError,
                      Group, HostSetup, Solver, lib, load_library)

__all__ = ["Solver", "Group", "HostSetup", "lib", "load_library", "CcmError", "CCM_FP64", "CCM_MIXED", "CCM_NONE",
           "CCM_DIRICHLET", "CCM_NEUMANN", "CCM_ROBIN"]
