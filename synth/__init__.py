"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This package holds no arithmetic of the filter itself.  It produces:

* ``sobol_params``  -- the Sobol generator parameters (primitive polynomials over
  GF(2) and initial direction integers, a stand-in for a published direction-number
  table) and the random affine-scramble draws (lower-triangular GF(2) matrices and
  digital shifts).  The recurrence that turns them into direction numbers, the
  Gray-code point construction and the scrambling are implemented separately by the
  oracle and by the CUDA path.
* ``trajectory``    -- Euler--Maruyama simulation of the filtering problem
  dX = f(X)dt + dV, dY = h(X)dt + dW (the problem statement of
  "Continuous-Time Nonlinear Filtering Problem"),
  producing the true states and the observation increments dy_k.
* ``configs``       -- the named workloads (sizes, step counts, seeds).

All random numbers come from numpy's Philox4x32-10 bit generator (Salmon et al.,
SC'11), seeded explicitly.
"""
from .configs import WORKLOADS, Workload, get_workload
from .sobol_params import sobol_poly_params, sobol_scramble_params, primitive_polynomials
from .trajectory import simulate, Trajectory

__all__ = [
    "WORKLOADS", "Workload", "get_workload",
    "sobol_poly_params", "sobol_scramble_params", "primitive_polynomials",
    "simulate", "Trajectory",
]
