"""FP64 CPU oracle for the THIIM E/H sweeps.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product package never imports,
links or executes anything here, and nothing here imports the product.

* ``thiim_oracle.c``  the 12 split updates as plain loop nests (Eqs. 3-7,
  Listings 1-2), compiled by ``build.py`` with gcc.
* ``coeffs.py``       the per-cell coefficient arrays t, c and the source
  arrays derived from Eqs. 3-5, in NumPy FP64.
  ``thiim_oracle.c`` also holds the adjoint of one iteration (reverse mode)
  with the coefficient gradients (``adjoint_steady`` sums it at a fixed
  point); ``coeffs.py`` the derivatives of the coefficients with respect to
  the real permittivity and the absorbed power.
"""
from .thiim_oracle import (iterate, adjoint_step, adjoint_steady, rule, SPLITS, FIELD_INDEX,  # noqa: F401
                           COEFF_NAMES)
from .coeffs import (build_coeffs, coeff_eps_derivatives, incident_wave, discrete_omega,  # noqa: F401
                     absorbed_power)
