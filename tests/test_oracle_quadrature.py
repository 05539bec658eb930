"""Pins for oracle/quadrature.py (Sec. 3.4: nu_j from a global quintic spline)."""
import numpy as np
import pytest
from scipy.interpolate import make_interp_spline

from oracle import grid
from oracle.quadrature import spline_weights


def _theta(L, t_max):
    return grid.theta_grid(L, grid.gamma_from_tmax(t_max))[0]


@pytest.mark.parametrize("L,t_max", [(17, 10.0), (129, 100.0), (513, 1e5)])
def test_exact_on_quintics(L, t_max):
    th = _theta(L, t_max)
    nu = spline_weights(th)
    for k in range(6):
        assert abs(nu @ th ** k - 1.0 / (k + 1)) < 1e-13


@pytest.mark.parametrize("L,t_max", [(33, 10.0), (129, 100.0)])
def test_matches_scipy_not_a_knot_quintic(L, t_max):
    th = _theta(L, t_max)
    ref = make_interp_spline(th, np.eye(L), k=5).integrate(0.0, 1.0)
    assert np.max(np.abs(spline_weights(th) - ref)) < 1e-14


def test_converges_on_smooth_integrand():
    """Against scipy's adaptive quad of a non-polynomial integrand: sixth-order decay."""
    from scipy.integrate import quad
    ref, _ = quad(lambda x: np.exp(np.sin(4 * x)), 0, 1, epsabs=1e-15, epsrel=1e-15)
    errs = []
    for L in [33, 65, 129]:
        th = _theta(L, 100.0)
        errs.append(abs(spline_weights(th) @ np.exp(np.sin(4 * th)) - ref))
    assert errs[1] < errs[0] / 16 and errs[2] < errs[1] / 16
