"""Quadrature weights nu_j of Sec. 3.4: integral over [0, 1] of a global quintic spline.

The paper fixes a quintic spline through (theta_j, g(theta_j)) and integrates it;
it does not state the end conditions. Reading: the not-a-knot quintic spline
(knots at theta_3 .. theta_{L-4} plus six-fold end knots, 0-based), so that

    sum_j nu_j g(theta_j) = integral_0^1 S[g](theta) dtheta.

Since S is linear in the data, nu = A^{-T} w where A is the B-spline collocation
matrix A[r, c] = B_c(theta_r) and w_c = integral of B_c = (t_{c+6} - t_c) / 6.
The B-splines come from the Cox-de Boor recursion; A is solved densely (slow,
plain and fine for an oracle).

Pins: tests/test_oracle_quadrature.py (sum nu = 1, exactness on theta^k for
k <= 5, agreement with scipy's make_interp_spline(k=5) integral, convergence on
a smooth non-polynomial integrand).
"""

import numpy as np

DEGREE = 5


def not_a_knot_knots(x, k=DEGREE):
    """Knot vector of the not-a-knot spline of odd degree k through sites x."""
    k2 = (k + 1) // 2
    inner = x[k2:-k2]
    return np.concatenate([np.full(k + 1, x[0]), inner, np.full(k + 1, x[-1])])


def bspline_matrix(knots, k, x):
    """B[r, c] = B_{c,k}(x_r) by the Cox-de Boor recursion (right end included)."""
    x = np.asarray(x, dtype=float)
    m = len(knots)
    # degree 0: indicator of [t_i, t_{i+1}); the right end point belongs to the
    # last non-empty interval.
    B = np.zeros((len(x), m - 1))
    last = max(i for i in range(m - 1) if knots[i] < knots[i + 1])
    for i in range(m - 1):
        if knots[i] < knots[i + 1]:
            B[:, i] = (knots[i] <= x) & (x < knots[i + 1])
    B[x == knots[-1], last] = 1.0
    for d in range(1, k + 1):
        Bn = np.zeros((len(x), m - 1 - d))
        for i in range(m - 1 - d):
            left = knots[i + d] - knots[i]
            right = knots[i + d + 1] - knots[i + 1]
            if left > 0:
                Bn[:, i] += (x - knots[i]) / left * B[:, i]
            if right > 0:
                Bn[:, i] += (knots[i + d + 1] - x) / right * B[:, i + 1]
        B = Bn
    return B


def spline_weights(theta):
    """nu_j such that sum_j nu_j g_j integrates the not-a-knot quintic spline."""
    theta = np.asarray(theta, dtype=float)
    L = len(theta)
    if L < DEGREE + 1:
        raise ValueError("need at least 6 grid points for a quintic spline")
    knots = not_a_knot_knots(theta)
    A = bspline_matrix(knots, DEGREE, theta)
    w = (knots[DEGREE + 1:] - knots[:L]) / (DEGREE + 1)
    return np.linalg.solve(A.T, w)
