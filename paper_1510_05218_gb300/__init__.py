"""GB300 THIIM E/H sweeps: a thin Python binding of libthiim.so.

Every step of the sweep runs in the library's CUDA kernels; this package only
marshals arguments (torch tensors -> device pointers, the current CUDA stream)
through the C ABI declared in include/thiim.h.  There is no CPU fallback:
importing the binding fails loudly when the library has not been built.
"""
from .thiim import (  # noqa: F401
    THIIM_C128, THIIM_C64, THIIM_C128_PAIR, THIIM_PERIODIC_X, THIIM_PERIODIC_Y, THIIM_PERIODIC_Z,
    THIIM_MAX_MATERIALS, THIIM_INT_ADD, THIIM_INT_MUL, THIIM_INT_SUMS, thiim_set_fp64_int_ops,
    ThiimError, lib_path, load_library, exported_symbols, declared_symbols,
    thiim_create, thiim_set_stream, thiim_set_tuning, thiim_set_coeffs, thiim_set_fields, thiim_iterate,
    thiim_residual, thiim_build_coeffs, thiim_mixed_solve, thiim_batch_iterate, thiim_adjoint_iterate, thiim_adjoint_steady, thiim_build_coeffs_grad,
    thiim_build_material_table, thiim_set_material_coeffs, thiim_build_coeffs_jones, thiim_absorbed_power,
    thiim_step_noalloc, thiim_fp64_pipe_rate, thiim_destroy, thiim_strerror, thiim_version,
    Solver,
)
