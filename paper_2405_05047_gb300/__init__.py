"""GB300 geometric-multigrid Krylov solver for adaptive Q1 finite elements.

Python binding of the C ABI declared in ``include/mg.h`` (argument
marshalling only; every step of a solve runs in the library's CUDA kernels).
The binding loads ``libmg_gb300.so`` built in-tree by ``build.py``; a missing
library or a missing GPU raises instead of falling back to anything else.
"""
from .binding import (MG_CG, MG_BICGSTAB, MG_ELASTICITY, MG_FP64, MG_GMRES, MG_KRYLOV_AUTO, MG_MIXED_FP32,
                      MG_OP_COARSE, MG_OP_MATVEC, MG_OP_PROLONG_ADD, MG_OP_RESTRICT, MG_OP_SMOOTH, MG_POISSON,
                      MG_TRANSPORT, Context, Hierarchy, MGError, NavierStokes, lib_path, load_library, mg_apply,
                      mg_assemble_rhs, mg_cancel, mg_destroy, mg_free, mg_hier_info, mg_init, mg_node_coords,
                      mg_poll, mg_serve_config, mg_setup, mg_solve, mg_solve_host, mg_solve_profiled, mg_submit,
                      mg_vcycle)

__all__ = [n for n in dir() if not n.startswith("_")]
