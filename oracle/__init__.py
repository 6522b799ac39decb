"""Plain, slow FP64 CPU oracle of the regularized-Bingham shallow-water DG method.

TEST INFRASTRUCTURE.  Only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package; the
library (``paper_2301_11238_gb300``) never does, and this package imports
nothing from the library.

Modules:
  refelem       quadrature, orthonormal modal bases, node sets
  constitutive  regularized Bingham stress (Sec. 4, Appendix A)
  dg            E-step, residual, mass solve, explicit SSP-RK3 (Sec. 3, Sec. 5)
  implicit      backward Euler + Newton with the Appendix A Jacobian (Sec. 5.1)
  riemann       exact shallow-water Riemann solution (Newtonian limit check)
  run           drivers that take a synthetic case and run it
"""
from .dg import Discretization  # noqa: F401
