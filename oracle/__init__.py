"""FP64 CPU oracle of the FR-SG scheme (arXiv 2112.05946).

TEST INFRASTRUCTURE.  Only the tests, the package smoke check and the CPU-baseline
leg of the benchmark may import this package.  It shares no code with the GPU
library: its tables, residual, filters, limiter and time stepping are written here
from the paper alone, in plain numpy FP64, step by step in the paper's order.

Modules
  tables     Gauss-Legendre points, Lagrange basis and derivative matrix, Radau
             correction functions, orthonormal Legendre gPC tables, Vandermonde.
  scheme     fluxes, local Lax-Friedrichs interface flux, 1D and 2D residual.
  capture    detector, exponential and L2 modal filters, positivity limiter.
  integrate  initial projection, CFL time step, SSP-RK3 stages, moments.

Every function is pinned by a test under tests/ that checks it against a closed
form, a library routine, an invariant or brute force; none is "parity unpinned".
"""
from . import capture, integrate, scheme, tables  # noqa: F401
from .scheme import Problem  # noqa: F401
