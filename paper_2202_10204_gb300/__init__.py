"""SPAI-GMRES-IR on one GB300 (sm_103a): sparse approximate inverse
preconditioning inside five-precision GMRES-based iterative refinement
(Carson & Khan, arXiv 2202.10204).

The numerical work lives in the CUDA library (``csrc/``, C ABI in
``include/spai_ir.h``); ``_lib`` is its ctypes binding and ``synth`` builds
seeded test systems.
"""
from ._lib import (ERR_ADMISSION, ERR_CUDA, ERR_INTERNAL, ERR_INVALID_ARG, ERR_NO_MEMORY, ERR_NONFINITE,
                   ERR_NOT_FOUND, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_ZERO_ROW, IR_CONVERGED, IR_STAGNATED,
                   IR_STOP_BACKWARD, IR_STOP_CORRECTION, IR_STOP_FIXED, OK, PENDING, SIDE_LEFT, SIDE_RIGHT,
                   WARN_FILLCAP, WARN_NOT_CONVERGED, Context, Precond, SpaiError, gmres_ir_solve,
                   gmres_ir_solve_batch, gmres_ir_solve_noalloc, make_ir_opts, make_spai_opts,
                   selftest_wait_timeout, solver_poll, solver_submit, spai_build, spai_build_batch, strerror,
                   tune_get, tune_set)

__all__ = ["ERR_ADMISSION", "ERR_CUDA", "ERR_INTERNAL", "ERR_INVALID_ARG", "ERR_NO_MEMORY", "ERR_NONFINITE",
           "ERR_NOT_FOUND", "ERR_TIMEOUT", "ERR_UNSUPPORTED", "ERR_ZERO_ROW", "IR_CONVERGED", "IR_STAGNATED",
           "IR_STOP_BACKWARD", "IR_STOP_CORRECTION", "IR_STOP_FIXED", "OK", "PENDING", "SIDE_LEFT", "SIDE_RIGHT",
           "WARN_FILLCAP", "WARN_NOT_CONVERGED", "Context", "Precond", "SpaiError", "gmres_ir_solve",
           "gmres_ir_solve_batch", "gmres_ir_solve_noalloc", "make_ir_opts", "make_spai_opts",
           "selftest_wait_timeout", "solver_poll", "solver_submit", "spai_build", "spai_build_batch", "strerror",
           "tune_get", "tune_set"]
