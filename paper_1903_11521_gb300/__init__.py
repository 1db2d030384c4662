"""yateto_gb300: GB300 (sm_103a) element kernels of tetrahedral ADER-DG, after
Uphoff & Bader, "Yet Another Tensor Toolbox for discontinuous Galerkin methods and other
applications" (arXiv 1903.11521).

The compute path is the in-tree shared library built from ``csrc/`` (C ABI in
``include/yateto_gb300.h``); this package only marshals arguments to it.  Importing the
package does not load the library; the first call that needs it does, and fails loudly
if it has not been built.
"""
from ._lib import (YT_BF16X3_F32ACC, YT_F32, YT_F64, YT_FIELD_DOFS, YT_FIELD_TIME_INTEGRAL, YT_MEM_DEVICE,
                   YT_MEM_HOST, YT_SCHEME_DIAG_EXPIRE_WAIT, YtError, load)
from .solver import Batch, Server, Solver, reference_matrix
from .plan import Plan, element_major, from_element_major

__all__ = ["Batch", "Server", "Plan", "element_major", "from_element_major", "Solver", "reference_matrix", "load", "YtError", "YT_F64", "YT_F32", "YT_BF16X3_F32ACC",
           "YT_MEM_HOST", "YT_MEM_DEVICE", "YT_FIELD_DOFS", "YT_FIELD_TIME_INTEGRAL", "YT_SCHEME_DIAG_EXPIRE_WAIT"]
