"""Seeded synthetic workloads for the THIIM E/H sweeps.

This package produces inputs only: per-cell relative permittivity maps of the
layered thin-film stack, absorbing-layer conductivity profiles, the TF/SF plane
wave description, and seeded random field/coefficient arrays.  It contains no
step of the iteration itself (no update coefficients, no stencil, no residual),
so both the CUDA path and the CPU oracle can take their inputs from here
without sharing any of the method's arithmetic.
"""
from .thiim_workloads import (  # noqa: F401
    N_FIELDS, N_COEFFS, MATERIALS, LayeredStack, stack_config, batch_configs,
    random_plane, random_fields, random_coeffs, random_sweep_inputs, WORKLOADS,
)
