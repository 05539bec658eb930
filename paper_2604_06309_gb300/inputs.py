"""Seeded synthetic inputs shaped like the paper's workloads (no solver arithmetic here).

A history is a set of slices t_0 = 0 < t_1 < ... with rows Cf, dCf/dt|theta, Rf,
dRf/dt|theta on a given theta grid. The fields below are smooth closed-form families
with the structure of an aging quench: a fast relaxation in the time difference
tau = t (1 - theta) near the diagonal, a slowly drifting plateau, Cf = Rf = 1 on the
diagonal and exact time derivatives at fixed theta:

    Cf(t, theta) = q(t) exp(-a tau) + (1 - q(t)) A(theta),   A = exp(-b w / (theta + c))
    Rf(t, theta) = exp(-a2 tau) [r(t) + (1 - r(t)) theta^kappa]
    q(t) = q0 + q1 / (1 + t),  r(t) = r0 + r1 / (1 + t),  w = 1 - theta

The parameters are drawn from numpy's default_rng(seed). Slice times are geometric
(the adaptive grid of a long run is close to geometric at late times) with t_0 = 0.
"""

import numpy as np


def geometric_times(n, t_first, t_last):
    """t_0 = 0 followed by n - 1 geometrically spaced times from t_first to t_last."""
    if n < 2:
        return np.zeros(1)
    return np.concatenate([[0.0], np.geomspace(t_first, t_last, n - 1)])


class SyntheticFields:
    def __init__(self, seed):
        rng = np.random.default_rng(seed)
        self.a, self.a2 = rng.uniform(0.5, 2.0, 2)
        self.q0, self.q1 = rng.uniform(0.5, 0.8), rng.uniform(0.0, 0.3)
        self.r0, self.r1 = rng.uniform(0.3, 0.6), rng.uniform(0.0, 0.3)
        self.b, self.c = rng.uniform(0.5, 2.0), rng.uniform(0.05, 0.5)
        self.kappa = rng.uniform(0.5, 2.0)

    def rows(self, t, theta, omega):
        """(C, dC, R, dR) at time t on the grid (theta, omega = 1 - theta)."""
        tau = t * omega
        q = self.q0 + self.q1 / (1.0 + t)
        dq = -self.q1 / (1.0 + t) ** 2
        r = self.r0 + self.r1 / (1.0 + t)
        dr = -self.r1 / (1.0 + t) ** 2
        ea = np.exp(-self.a * tau)
        A = np.exp(-self.b * omega / (theta + self.c))
        C = q * ea + (1.0 - q) * A
        dC = dq * (ea - A) - self.a * omega * q * ea
        B = theta ** self.kappa
        e2 = np.exp(-self.a2 * tau)
        R = e2 * (r + (1.0 - r) * B)
        dR = -self.a2 * omega * R + e2 * dr * (1.0 - B)
        C[-1] = R[-1] = 1.0
        dC[-1] = dR[-1] = 0.0
        return C, dC, R, dR

    def history(self, times, theta, omega):
        """Rows for every slice time: four arrays of shape [len(times), L]."""
        rows = [self.rows(t, theta, omega) for t in times]
        return tuple(np.array([r[k] for r in rows]) for k in range(4))


def synthetic_history(seed, times, theta, omega):
    return SyntheticFields(seed).history(times, theta, omega)


# Workload shapes (Sec. 4.1 runs: mixed (3+4)-spin, lambda = 1/2, quench; grids of the
# benchmark configurations).
MIXED_34 = {3: 0.25, 4: 0.25}       # f(q) = (lambda q^3 + (1 - lambda) q^4) / 2, lambda = 1/2
PURE_3 = {3: 0.5}                   # f(q) = q^3 / 2
