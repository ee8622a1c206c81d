"""GB300-native matrix-free phase-field fracture solver (sm_103a CUDA behind a C-ABI).

Public entry points mirror the C library ``libpff`` (include/pff.h): ``setup_mesh`` returns a
``Context`` whose methods are ``set_state``, ``apply_jacobian``, ``residual``, ``vcycle``,
``solve_newton_step`` and friends, and ``ResidualFunction`` wraps the residual in
``torch.autograd`` with the hand-written adjoint. The CUDA library is loaded on first use;
there is no CPU fallback.
"""
from .pff import (  # noqa: F401
    PFF_ERR_BREAKDOWN, PFF_ERR_CUDA, PFF_ERR_INVALID_ARG, PFF_ERR_NAN, PFF_ERR_NO_STATE, PFF_ERR_NOT_CONVERGED,
    PFF_ERR_OOM, PFF_ERR_TOO_LARGE, PFF_ERR_UNAVAILABLE, PFF_OK,
    PFF_FLAG_BOTTOM, PFF_FLAG_COPY, PFF_FLAG_SLIT, PFF_FLAG_TOP, PFF_MASK_ADJOINT, PFF_MASK_RAW, PFF_MODE_BLOCKDIAG,
    PFF_MODE_FULL, PFF_MODE_TRANSPOSE, PFF_PROF_JAC32, PFF_PROF_JAC32_L0, PFF_PROF_JAC64,
    PFF_PROF_JAC64_L0, PFF_PROF_OFF, PFF_PROF_RESIDUAL, PFF_SPLIT_MIEHE, PFF_SPLIT_NONE, Context, PFFError, ResidualFunction,
    csr_pattern, csr_probe_targets, default_params, launch_count, load_library, report_lines, setup_mesh)
