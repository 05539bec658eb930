"""Plain FP64 CPU oracle for the DMFE history-integral path (DYNAMITE, arXiv 2604.06309).

This package is TEST INFRASTRUCTURE. Only the test suite, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` import it. The CUDA
library never calls it and shares no code, tables or constants with it.

Every function restates the paper's method in straightforward numpy, following
the section or equation named in its docstring:

* ``grid``        Sec. 3.2, Eq. (theta): the theta grid, gamma = -W_{-1}(-1/t_max),
                  the inverse map theta -> fractional index.
* ``interp``      Sec. 3.3: index-space Lagrange stencils and cubic Hermite in t.
* ``quadrature``  Sec. 3.4: the weights nu_j of a global quintic spline.
* ``model``       Sec. 2.1: f(q) = sum_p c_p q^p and its derivatives.
* ``integrals``   Secs. 2.1, 3.3, 3.4, Eqs. (genericDMFE), (int): the history
                  integrals, mu(t), E(t) and the right-hand side.
* ``solver``      Secs. 3.1, 3.5, 3.6: Dormand-Prince 5(4), the step-control
                  rule, the history store, rollback and sparsification.
* ``closed_forms`` independent reference solutions used only as pins: the pure
                  p=2 model at T=0, the equilibrium (TTI + FDT) one-time equation
                  above T_d and a brute-force uniform-grid two-time solver.

Parity status of each function is listed in the module docstrings; every one is
pinned by a ``-m "not gpu"`` test in ``tests/test_oracle_*.py``.
"""

from . import grid, interp, quadrature, model, integrals, solver, closed_forms  # noqa: F401
