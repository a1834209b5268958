"""GB300 CUDA implementation of the graph-based AMG for hierarchical-P2 systems.

The solver lives in the C-ABI library libamgp2.so (include/amgp2.h), built by
`paper_1503_01287_gb300.build.build()`; `binding` marshals arguments to it.
"""
from .binding import (AMG_FP32, AMG_FP64, AMG_KRYLOV_AUTO, AMG_KRYLOV_FCG,  # noqa: F401
                      AMG_KRYLOV_FGMRES, AMG_KRYLOV_NONE, AMG_KRYLOV_PCG, AMG_SMOOTHER_GS,
                      AMG_SMOOTHER_JACOBI, AMG_SMOOTHER_SGS, AmgError, Handle, default_options,
                      load_library, setup_problem)
