"""Theta grid of Sec. 3.2, Eq. (theta), and its inverse.

The grid is theta(i), i = 1..L:

    theta(i) = [atan(e^gamma) - atan(e^{-gamma y(z(i))})] / [atan(e^gamma) - atan(e^{-gamma})]
    y(z)     = (2 z - 1 - L) / (L - 1)
    z(i)     = alpha * phi_delta(i) + (1 - alpha) * i
    phi_delta(i) = (L-1)/2 * (g_delta(y(i)) / g_delta(1) + 1) + 1
    gamma    = -W_{-1}(-1 / t_max)

Readings (Eq. theta is garbled for delta > 0): g_delta is taken odd,
g_delta(x) = sign(x) [(|x|^3 + delta^3)^{1/3} - delta], so that theta(1) = 0 and
theta(L) = 1 for every alpha, delta.

With a = atan(e^{-gamma}) and D = atan(e^gamma) - a the numerator can be written
atan(e^{gamma y}) - a, which is how it is evaluated here (the same number, without
the cancellation near theta = 0); the complement 1 - theta is theta(-y) because the
grid is symmetric about theta = 1/2. Both theta and 1 - theta are kept, since
t (1 - theta) is a physical time difference near the diagonal.

Pins: tests/test_oracle_grid.py (Lambert W against scipy, symmetry, endpoints,
round trip of the inverse, the grid condition Eq. (condition)).
"""

import numpy as np


def gamma_from_tmax(t_max):
    """gamma = -W_{-1}(-1/t_max): the root gamma > 1 of gamma e^{-gamma} = 1/t_max.

    Needs t_max > e (for t_max <= e the lower branch is not defined there).
    Solved by bisection on ln(gamma) - gamma + ln(t_max) = 0, then Newton.
    """
    t_max = float(t_max)
    if not t_max > np.e:
        raise ValueError("grid t_max must exceed e for the W_{-1} branch")
    lt = np.log(t_max)
    g = lambda x: np.log(x) - x + lt  # decreasing on x > 1, g(1) > 0
    lo, hi = 1.0, 2.0 * lt + 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if g(mid) > 0:
            lo = mid
        else:
            hi = mid
    x = 0.5 * (lo + hi)
    for _ in range(3):
        x = x - g(x) / (1.0 / x - 1.0)
    return x


def _g_delta(x, delta):
    return np.sign(x) * (np.cbrt(np.abs(x) ** 3 + delta ** 3) - delta)


def z_of_i(i, L, alpha, delta):
    """z_(alpha,delta)(i) of Eq. (theta) (i is 1-based and may be fractional)."""
    i = np.asarray(i, dtype=float)
    if alpha == 0.0 or delta == 0.0:
        # phi_delta(i) = i when delta = 0, so z = i.
        return i.copy()
    y = (2.0 * i - 1.0 - L) / (L - 1.0)
    phi = 0.5 * (L - 1.0) * (_g_delta(y, delta) / _g_delta(1.0, delta) + 1.0) + 1.0
    return alpha * phi + (1.0 - alpha) * i


def _theta_of_y(y, gamma):
    # [atan(e^{gamma y}) - atan(e^{-gamma})] / D, written as one atan of a quotient.
    a = np.arctan(np.exp(-gamma))
    D = np.arctan(np.exp(gamma)) - a
    num = np.exp(-gamma) * np.expm1(gamma * (y + 1.0))
    den = 1.0 + np.exp(gamma * (y - 1.0))
    return np.arctan(num / den) / D


def theta_grid(L, gamma, alpha=0.0, delta=0.0):
    """Return (theta, omega = 1 - theta) on the L grid points of Eq. (theta)."""
    if L < 8:
        raise ValueError("L must be at least 8")
    i = np.arange(1, L + 1, dtype=float)
    y = (2.0 * z_of_i(i, L, alpha, delta) - 1.0 - L) / (L - 1.0)
    theta = _theta_of_y(y, gamma)
    omega = _theta_of_y(-y, gamma)
    theta[0], omega[0] = 0.0, 1.0
    theta[-1], omega[-1] = 1.0, 0.0
    return theta, omega


def _i_of_z(z, L, alpha, delta):
    """Invert z(i) of Eq. (theta) (monotone in i) by bisection on [1, L]."""
    z = np.asarray(z, dtype=float)
    if alpha == 0.0 or delta == 0.0:
        return z.copy()
    lo = np.ones_like(z)
    hi = np.full_like(z, float(L))
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        below = z_of_i(mid, L, alpha, delta) < z
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    return 0.5 * (lo + hi)


def frac_index(th, om, L, gamma, alpha=0.0, delta=0.0):
    """0-based fractional grid index x with theta(x + 1) = th (inverse of Eq. theta).

    ``om`` must hold 1 - th computed without cancellation; the branch th > 1/2
    works from it. With alpha = 0 (or delta = 0) the inverse is closed form:
    y = ln tan(a + th D) / gamma, x = (L - 1)(y + 1)/2.
    """
    th = np.asarray(th, dtype=float)
    om = np.asarray(om, dtype=float)
    a = np.arctan(np.exp(-gamma))
    D = np.arctan(np.exp(gamma)) - a
    lower = th <= 0.5
    arg = np.where(lower, a + th * D, a + om * D)
    y = np.log(np.tan(arg)) / gamma
    y = np.where(lower, y, -y)
    z = 0.5 * (y * (L - 1.0) + 1.0 + L)
    x = _i_of_z(z, L, alpha, delta) - 1.0
    return np.clip(x, 0.0, L - 1.0)
