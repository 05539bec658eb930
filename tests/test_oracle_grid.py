"""Pins for oracle/grid.py (Sec. 3.2, Eq. theta)."""
import numpy as np
import pytest
from scipy.special import lambertw

from oracle import grid


@pytest.mark.parametrize("t_max", [3.0, 100.0, 1e5, 1e7])
def test_gamma_is_lambert_w_lower_branch(t_max):
    g = grid.gamma_from_tmax(t_max)
    assert g > 1.0
    assert abs(g - (-lambertw(-1.0 / t_max, -1).real)) < 1e-12 * g
    assert abs(g * np.exp(-g) * t_max - 1.0) < 1e-14


def test_gamma_rejects_small_tmax():
    with pytest.raises(ValueError):
        grid.gamma_from_tmax(2.0)


@pytest.mark.parametrize("L,t_max", [(33, 10.0), (129, 100.0), (2049, 1e5)])
def test_theta_matches_printed_formula(L, t_max):
    """The rewritten atan difference equals Eq. (theta) as printed (alpha = 0)."""
    g = grid.gamma_from_tmax(t_max)
    th, om = grid.theta_grid(L, g)
    i = np.arange(1, L + 1)
    y = (2 * i - 1 - L) / (L - 1)
    printed = (np.arctan(np.exp(g)) - np.arctan(np.exp(-g * y))) / (np.arctan(np.exp(g)) - np.arctan(np.exp(-g)))
    assert np.max(np.abs(th - printed)) < 1e-14
    assert th[0] == 0.0 and th[-1] == 1.0
    assert np.all(np.diff(th) > 0)
    # symmetric grid: 1 - theta(i) = theta(L + 1 - i), and omega is that complement
    assert np.max(np.abs(om - th[::-1])) < 1e-16
    assert np.max(np.abs(th + om - 1.0)) < 2.3e-16


def test_complement_is_accurate_near_the_diagonal():
    """omega keeps full relative precision where 1 - theta would cancel."""
    g = grid.gamma_from_tmax(1e7)
    th, om = grid.theta_grid(4097, g)
    # near theta = 1 the spacing is ~1e-10: compare with an extended-precision evaluation
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    i = 4096 - 1  # last interior point (1-based 4096)
    y = mp.mpf(2 * (i + 1) - 1 - 4097) / 4096
    gm = mp.mpf(g)
    exact = 1 - (mp.atan(mp.e ** gm) - mp.atan(mp.e ** (-gm * y))) / (mp.atan(mp.e ** gm) - mp.atan(mp.e ** (-gm)))
    assert abs(om[i] - float(exact)) < 1e-14 * float(exact)


@pytest.mark.parametrize("alpha,delta", [(0.0, 0.0), (0.5, 0.2), (0.8, 0.3)])
def test_frac_index_round_trip(alpha, delta):
    L = 257
    g = grid.gamma_from_tmax(1e4)
    th, om = grid.theta_grid(L, g, alpha, delta)
    assert th[0] == 0.0 and th[-1] == 1.0 and np.all(np.diff(th) > 0)
    x = grid.frac_index(th, om, L, g, alpha, delta)
    assert np.max(np.abs(x - np.arange(L))) < 1e-9


def test_grid_condition_at_t_max():
    """Eq. (condition): theta spacing << tau_micro / t near both ends at t = t_max."""
    for L, t_max in [(129, 100.0), (2049, 1e5), (4097, 1e7)]:
        g = grid.gamma_from_tmax(t_max)
        th, om = grid.theta_grid(L, g)
        d = np.diff(th)
        assert t_max * d[0] < 0.05 and t_max * d[-1] < 0.05
