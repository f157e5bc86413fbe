"""GB300 (sm_103a) CTENO / CTENOZ finite-volume solver for the compressible Euler equations on
triangle and tetrahedron meshes (arXiv 2312.17042).

The compute path is the CUDA library ``libcteno.so`` (C ABI in include/cteno.h); this package
only marshals arguments to it. Importing the package does not load the library; the first call
does, and raises if the library has not been built (``python -m paper_2312_17042_gb300.build``).
There is no CPU fallback.
"""
from .native import (  # noqa: F401
    CTENO_FP64, CTENO_MIXED, CTENO_SCHEME_CTENO, CTENO_SCHEME_CTENOZ, CtenoError, Solver,
    cteno_autotune, cteno_create, cteno_default_params, cteno_destroy, cteno_get_dt,
    cteno_get_face_states, cteno_get_flags, cteno_get_state, cteno_get_state_noalloc, cteno_get_stencil, cteno_info,
    cteno_kernel_stats, cteno_last_error, cteno_last_kernel_ms, cteno_measure_alu_peak, cteno_set_timing, cteno_lsq_build, cteno_mesh_build, cteno_params,
    cteno_profile_step, cteno_record_flags, cteno_rk_stage, cteno_run, cteno_set_launch,
    cteno_set_state, cteno_stencil_build, cteno_sync, library_path, load_library,
)
