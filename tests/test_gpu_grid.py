"""GPU (kernel a and host grid) against the oracle: theta, nu and the stencil positions."""
import numpy as np
import pytest

from gpu_common import need_gpu
from oracle import integrals as OI

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L,t_max,alpha,delta", [(33, 10.0, 0.0, 0.0), (129, 100.0, 0.0, 0.0),
                                                  (257, 1e4, 0.5, 0.2), (2049, 1e5, 0.0, 0.0)])
def test_grid_and_weights(L, t_max, alpha, delta):
    need_gpu()
    from paper_2604_06309_gb300 import Solver
    sv = Solver({3: 0.5}, 0.8, L, t_max, alpha=alpha, delta=delta, history_cap=16)
    G = OI.Grid(L, t_max, alpha=alpha, delta=delta) if L <= 257 else None
    from oracle import grid as og, quadrature as oq
    gam = og.gamma_from_tmax(t_max)
    th, om = og.theta_grid(L, gam, alpha, delta)
    assert np.max(np.abs(sv.theta - th)) < 2e-16
    assert np.max(np.abs(sv.omega - om) / np.maximum(om, 1e-300)) < 1e-14
    nu = G.nu if G is not None else oq.spline_weights(th)
    assert np.max(np.abs(sv.nu - nu)) < 1e-13 * max(1.0, np.max(np.abs(nu)) * L)
    sv.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "df"])
@pytest.mark.parametrize("L,t_max,alpha,delta", [(129, 100.0, 0.0, 0.0), (97, 1e4, 0.5, 0.2)])
def test_stencil_tables(precision, L, t_max, alpha, delta):
    need_gpu()
    from paper_2604_06309_gb300 import Solver
    sv = Solver({3: 0.5}, 0.8, L, t_max, alpha=alpha, delta=delta, history_cap=16, precision=precision)
    x1, x2, x3 = sv.tables()
    G = OI.Grid(L, t_max, alpha=alpha, delta=delta)
    _, r1, r2, r3 = G.positions(slice(0, L))[:4]
    tol = 1e-9 if precision == "fp64" else 2.0 ** -20 + 1e-9
    for a, b in ((x1, r1), (x2, r2), (x3, r3)):
        assert np.max(np.abs(a - b)) < tol
        # the integer stencil cell agrees wherever x is not within rounding of an integer
        far = np.abs(b - np.round(b)) > 1e-6
        assert np.array_equal(np.floor(a[far]), np.floor(b[far]))
    sv.close()
