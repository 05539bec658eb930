"""Adaptive Runge-Kutta driver, step control, rollback and sparsification.

Secs. 3.1 (the step recipe), 3.5 (adaptive ODE solver) and 3.6 (selective history
reduction). Readings where the paper is silent:

* Integrators (Sec. 3.5): Dormand-Prince 5(4) at early times, then the ten-stage
  fourth-order strong-stability-preserving method SSPRK(10,4) of Ketcheson (2008).
  Its Butcher form is generated here from the published low-storage recurrence
  (five Euler substeps of h/6, the register combination 1/25, 9/25 and 15, -5, four
  more substeps, final update with h/10). The paper names no embedded estimate for
  it; the one used here is the third-order weight vector of minimal 2-norm on the
  same ten stages whose last weight is zero (exactly third order, all weights >= 0).
* Switch (Sec. 3.5): the spectrum of the Jacobian lies on the negative real axis
  within radius 4 sqrt(f''(1)). After an accepted Dormand-Prince step whose new
  controller step dt reaches beta_DP / (4 sqrt(f''(1))), with beta_DP the length of
  the real stability interval of Dormand-Prince 5, the method becomes SSPRK(10,4)
  and dt is halved. There is no switch back (a rollback keeps the current method).

* Step rule (Sec. 3.5): eps_RK = sum_i |dC_i| + |dR_i| from the embedded 4th-order
  estimate. eps_RK > 2 tol: reject, revert the last min(10, N-1) stored slices and
  halve dt. Otherwise accept; then dt *= 0.9 if eps_RK > tol, dt *= 1.01 if
  eps_RK < tol/2. dt < dt_min ends the run with status "step underflow" (App. B).
  The last step is shortened to land on t_max.
* The stored derivative of a slice is the right-hand side at that slice (DP's
  FSAL stage k7), so k1 of the next step is the stored derivative.
* Sparsification (Sec. 3.6): candidates n = 1 .. N-12 (slice 0, the last slice
  and the 10-slice rollback window are kept). eps_sparse(n) = sum_i |Delta^C| +
  |Delta^R| with Delta the difference of the integrals over [t_{n-1}, t_{n+1}] of
  the Hermite interpolants with and without slice n. Scanning n upwards, n is
  removed if eps_sparse(n) < tol/10, and then n+1 is skipped. A pass runs when
  the store is full; if it frees nothing, the candidate with the smallest
  eps_sparse is removed and counted as forced.

Pins: tests/test_oracle_solver.py (DP5 and SSPRK(10,4) order and error-estimate
order on scalar ODEs, exact order conditions of the generated tableau, the
low-storage recurrence reproduced step by step, the DP5 stability polynomial and
its real stability interval by direct one-step amplification, the p = 2 energy against the closed form, f = 0 exact solution, agreement
with the brute-force uniform-grid solver, equilibrium FDT above T_d, the Hermite
integral identity and cubic slices being removed by sparsification).
"""

import numpy as np

from .integrals import Grid, History, rhs
from .interp import lagrange_stencil, hermite, hermite_integral
from . import grid as gridmod

# Dormand & Prince (1980) RK5(4)7M tableau.
DP_C = np.array([0.0, 1 / 5, 3 / 10, 4 / 5, 8 / 9, 1.0, 1.0])
DP_A = [
    [],
    [1 / 5],
    [3 / 40, 9 / 40],
    [44 / 45, -56 / 15, 32 / 9],
    [19372 / 6561, -25360 / 2187, 64448 / 6561, -212 / 729],
    [9017 / 3168, -355 / 33, 46732 / 5247, 49 / 176, -5103 / 18656],
    [35 / 384, 0.0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84],
]
DP_B5 = np.array([35 / 384, 0.0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84, 0.0])
DP_B4 = np.array([5179 / 57600, 0.0, 7571 / 16695, 393 / 640, -92097 / 339200, 187 / 2100, 1 / 40])
DP_E = DP_B5 - DP_B4

OK, ERR_STEP_UNDERFLOW, ERR_CAPACITY, ERR_NONFINITE = 0, -4, -5, -3


class RKMethod:
    """Explicit Runge-Kutta pair in first-same-as-last form.

    Stage 0 is f at the start of the step (the stored derivative). Stages 1..n are
    evaluated at t + c[st] h on Y_st = y + h sum_{l < st} A[st][l] k_l; row A[n] is
    the propagating weight vector b, so Y_n is the new solution and k_n = f(t + h,
    Y_n) its derivative. The error estimate is h sum_l E[l] k_l over l = 0..n.
    """

    def __init__(self, name, c, A, E):
        self.name = name
        self.n = len(A) - 1
        self.c = np.asarray(c, dtype=float)
        self.A = [[float(a) for a in row] for row in A]
        self.E = np.asarray(E, dtype=float)


def ssprk104_exact():
    """SSPRK(10,4) Butcher coefficients (exact fractions) from its low-storage form.

    Returns (c, A, b, bhat) for the ten method stages (0-based, stage 0 at the step
    start), with bhat the embedded third-order weights described in the module
    docstring. Each register holds its coefficients on (y, h k_0, ..., h k_9).
    """
    from fractions import Fraction as Fr
    ns = 10
    one = [Fr(1)] + [Fr(0)] * ns

    def axpy(a, x, b_, y):
        return [a * xi + b_ * yi for xi, yi in zip(x, y)]

    rows = []
    q1, q2 = list(one), list(one)

    def euler(q, weight):
        st = len(rows)
        rows.append(q)
        q = list(q)
        q[1 + st] += weight
        return q

    for _ in range(5):
        q1 = euler(q1, Fr(1, 6))
    q2 = axpy(Fr(1, 25), q2, Fr(9, 25), q1)
    q1 = axpy(Fr(15), q2, Fr(-5), q1)
    for _ in range(4):
        q1 = euler(q1, Fr(1, 6))
    # final update u = q2 + 3/5 q1 + h/10 f(q1)
    rows.append(q1)
    new = axpy(Fr(1), q2, Fr(3, 5), q1)
    new[1 + 9] += Fr(1, 10)
    A = [[r[1 + l] for l in range(st)] for st, r in enumerate(rows)]
    c = [sum(a) for a in A]
    b = [new[1 + l] for l in range(ns)]
    assert all(r[0] == 1 for r in rows) and new[0] == 1
    bhat = [Fr(3, 20), Fr(1, 12), Fr(7, 120), Fr(3, 40), Fr(2, 15), Fr(7, 120), Fr(3, 40), Fr(2, 15),
            Fr(7, 30), Fr(0)]
    return c, A, b, bhat


def _ssprk104():
    c, A, b, bhat = ssprk104_exact()
    rows = [list(r) for r in A] + [list(b)]
    cc = list(c) + [1]
    E = [bi - bh for bi, bh in zip(b, bhat)] + [0]
    return RKMethod("ssprk104", [float(x) for x in cc], rows, [float(x) for x in E])


DP5 = RKMethod("dp5", DP_C, DP_A, DP_E)
SSPRK104 = _ssprk104()
METHODS = {"dp5": DP5, "ssprk104": SSPRK104}


def stability_coefficients(method):
    """gamma_k with R(z) = 1 + sum_k gamma_k z^k, gamma_k = b^T A^{k-1} 1 (stages 0..n-1)."""
    n = method.n
    A = np.zeros((n, n))
    for st in range(n):
        A[st, :st] = method.A[st][:st] if st > 0 else []
    b = np.asarray(method.A[n][:n], dtype=float)
    g, v = [1.0], np.ones(n)
    for _ in range(n):
        g.append(float(b @ v))
        v = A @ v
    return np.array(g)


def real_stability_boundary(method):
    """Largest x with |R(-y)| <= 1 for all y in [0, x] (scan, then bisection)."""
    g = stability_coefficients(method)
    R = lambda y: abs(np.polyval(g[::-1], -y))
    y, dy = 0.0, 1e-3
    while R(y + dy) <= 1.0 + 1e-14:
        y += dy
        if y > 1e3:
            return np.inf
    lo, hi = y, y + dy
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if R(mid) <= 1.0:
            lo = mid
        else:
            hi = mid
    return lo


DP5_REAL_STABILITY = real_stability_boundary(DP5)


def switch_dt_auto(model):
    """dt at which Dormand-Prince 5 meets its stability limit (Sec. 3.5): the
    Jacobian's spectral radius is at most 4 sqrt(f''(1)); inf if f''(1) <= 0."""
    fpp1 = float(model.fpp(1.0))
    if fpp1 <= 0.0:
        return np.inf
    return DP5_REAL_STABILITY / (4.0 * np.sqrt(fpp1))


def rk_step(method, f, t, y, h, k0):
    """One step of an RKMethod; returns (y_new, err, ks) with ks[n] = f(t + h, y_new)."""
    ks = [k0]
    yk = y
    for st in range(1, method.n + 1):
        yk = y + h * sum(method.A[st][l] * ks[l] for l in range(st))
        ks.append(f(t + method.c[st] * h, yk))
    err = h * sum(method.E[l] * ks[l] for l in range(method.n + 1))
    return yk, err, ks


def dp5_step(f, t, y, h, k1):
    """One Dormand-Prince 5(4) step of y' = f(t, y) with k1 = f(t, y) given (FSAL).

    Returns (y_new, err, ks): the 5th-order solution, the embedded error estimate
    h * sum_l e_l k_l and the seven stage derivatives (ks[6] = f(t + h, y_new)).
    """
    ks = [k1]
    for st in range(1, 7):
        yk = y + h * sum(DP_A[st][l] * ks[l] for l in range(st))
        ks.append(f(t + DP_C[st] * h, yk))
    y_new = y + h * sum(DP_B5[l] * ks[l] for l in range(7))
    err = h * sum(DP_E[l] * ks[l] for l in range(7))
    return y_new, err, ks


def sparsify_residuals(hist):
    """eps_sparse(n) for every slice n = 1 .. N-2 (Sec. 3.6); entry n of the result."""
    t = hist.t
    N = hist.N
    eps = np.full(N, np.inf)
    for n in range(1, N - 1):
        h1, h2 = t[n] - t[n - 1], t[n + 1] - t[n]
        tot = 0.0
        for Y, dY in ((hist.C, hist.dC), (hist.R, hist.dR)):
            with_n = hermite_integral(Y[n - 1], dY[n - 1], Y[n], dY[n], h1) + \
                hermite_integral(Y[n], dY[n], Y[n + 1], dY[n + 1], h2)
            without = hermite_integral(Y[n - 1], dY[n - 1], Y[n + 1], dY[n + 1], h1 + h2)
            tot += np.sum(np.abs(with_n - without))
        eps[n] = tot
    return eps


def sparsify_pass(hist, tol, stats=None, force=True):
    """One pass of Sec. 3.6; returns (thinned history, whether the pass ran). A pass runs
    when there is at least one candidate (slices 1 .. N-12). force: when no candidate
    qualifies, remove the one with the smallest residual (a pass on a full store must
    free a slot); without it such a pass removes nothing."""
    N = hist.N
    last = N - 12
    if last < 1:
        return hist, False
    eps = sparsify_residuals(hist)
    keep = np.ones(N, dtype=bool)
    n = 1
    removed = 0
    while n <= last:
        if eps[n] < tol / 10.0:
            keep[n] = False
            removed += 1
            if stats is not None:
                stats["max_eps_sparse"] = max(stats["max_eps_sparse"], eps[n])
            n += 2
        else:
            n += 1
    if removed == 0 and force:
        m = 1 + int(np.argmin(eps[1:last + 1]))
        keep[m] = False
        removed = 1
        if stats is not None:
            stats["forced_removals"] += 1
            stats["max_eps_sparse"] = max(stats["max_eps_sparse"], eps[m])
    if stats is not None:
        stats["sparsify_passes"] += 1
        stats["slices_removed"] += removed
    return hist.keep(keep), True


class Solver:
    """Plain FP64 solver state: grid, model, history and step control."""

    def __init__(self, coefs, T, L, grid_t_max, s=4, beta0=0.0, alpha=0.0, delta=0.0,
                 history_cap=None, dt0=1e-4, dt_min=1e-12, sparsify=True, integrator="auto",
                 switch_dt=0.0, interp="lagrange_index", fh_d=3, log_r=False, sparsify_every=0,
                 sparsify_passes=1):
        """integrator: "dp5" (Dormand-Prince throughout), "ssprk104" (SSPRK(10,4)
        throughout) or "auto" (Dormand-Prince, then SSPRK(10,4) once dt reaches
        switch_dt; switch_dt = 0 takes the stability estimate switch_dt_auto).

        Sparsification (Sec. 3.6; the user sets the number of passes, reading R16): a
        round of sparsify_passes passes runs whenever the store is full (sparsify=True)
        and, if sparsify_every = P > 0, after every P-th accepted step. The first pass of
        a full-store round may force a removal; the accepted slice is appended after it,
        before the round's further passes. A periodic round runs after the append."""
        from .model import Model
        self.model = Model(coefs, T, beta0)
        self.grid = Grid(L, grid_t_max, s, alpha, delta, interp=interp, fh_d=fh_d, log_r=log_r)
        self.cap = int(history_cap if history_cap is not None else L)
        if self.cap < 16:
            raise ValueError("history_cap must be at least 16")
        self.dt = float(dt0)
        self.dt_min = float(dt_min)
        self.sparsify = sparsify
        self.sparsify_every = int(sparsify_every)
        self.sparsify_passes = max(1, int(sparsify_passes))
        if integrator not in ("dp5", "ssprk104", "auto"):
            raise ValueError("integrator must be dp5, ssprk104 or auto")
        self.integrator = integrator
        self.method = SSPRK104 if integrator == "ssprk104" else DP5
        self.switch_dt = (switch_dt_auto(self.model) if switch_dt == 0.0 else float(switch_dt)) \
            if integrator == "auto" else np.inf
        self.t_switch = None
        ones = np.ones(L)
        dC0, dR0, mu0, E0 = rhs(self.model, self.grid, None, 0.0, ones, ones)
        self.hist = History([0.0], ones[None, :], dC0[None, :], ones[None, :], dR0[None, :])
        self.mu, self.E = mu0, E0
        self.stats = dict(steps_accepted=0, steps_rejected=0, rhs_evals=0, sparsify_passes=0,
                          slices_removed=0, forced_removals=0, max_eps_sparse=0.0)
        self.log = []  # (t, h, eps_RK, accepted)

    @property
    def t(self):
        return self.hist.t[-1]

    def _f(self, t, y):
        L = self.grid.L
        dC, dR, _, _ = rhs(self.model, self.grid, self.hist, t, y[:L], y[L:])
        self.stats["rhs_evals"] += 1
        return np.concatenate([dC, dR])

    def step(self, h):
        """Trial step of size h from the last slice with the current method; returns
        (y_new, derivative at y_new, eps_RK)."""
        y = np.concatenate([self.hist.C[-1], self.hist.R[-1]])
        k0 = np.concatenate([self.hist.dC[-1], self.hist.dR[-1]])
        if self.method is DP5:
            y_new, err, ks = dp5_step(self._f, self.t, y, h, k0)
        else:
            y_new, err, ks = rk_step(self.method, self._f, self.t, y, h, k0)
        return y_new, ks[-1], float(np.sum(np.abs(err)))

    def integrate(self, t_max, tol):
        """Advance to t_max (Secs. 3.1, 3.5, 3.6); returns a status code."""
        L = self.grid.L
        while self.t < t_max:
            h = min(self.dt, t_max - self.t)
            t0 = self.t
            y_new, k7, eps = self.step(h)
            if not np.isfinite(eps):
                return ERR_NONFINITE
            if eps > 2.0 * tol:
                self.log.append((t0, h, eps, False))
                self.stats["steps_rejected"] += 1
                drop = min(10, self.hist.N - 1)
                self.hist = self.hist.keep(np.arange(self.hist.N) < self.hist.N - drop)
                self.dt *= 0.5
            else:
                self.log.append((t0, h, eps, True))
                self.stats["steps_accepted"] += 1
                passes = 0
                if self.hist.N >= self.cap:
                    if not self.sparsify:
                        return ERR_CAPACITY
                    self.hist, ran = sparsify_pass(self.hist, tol, self.stats)
                    if not ran:
                        return ERR_CAPACITY
                    passes = self.sparsify_passes - 1
                elif self.sparsify_every > 0 and self.stats["steps_accepted"] % self.sparsify_every == 0:
                    passes = self.sparsify_passes
                t1 = t0 + h if h < t_max - t0 else t_max
                self.hist = self.hist.append(t1, y_new[:L], k7[:L], y_new[L:], k7[L:])
                for _ in range(passes):
                    self.hist, _ = sparsify_pass(self.hist, tol, self.stats, force=False)
                if eps > tol:
                    self.dt *= 0.9
                elif eps < 0.5 * tol:
                    self.dt *= 1.01
                if self.method is DP5 and self.dt >= self.switch_dt:
                    self.method = SSPRK104
                    self.dt *= 0.5
                    self.t_switch = t1
            if self.dt < self.dt_min:
                return ERR_STEP_UNDERFLOW
        C, R = self.hist.C[-1], self.hist.R[-1]
        from .integrals import row_prep
        _, _, self.mu, self.E = row_prep(self.model, self.grid, self.t, C, R)
        return OK

    def get_C(self, t, tp):
        return get_two_time(self.grid, self.hist, t, tp, "C")

    def get_R(self, t, tp):
        return get_two_time(self.grid, self.hist, t, tp, "R")


def get_two_time(grid, hist, t, tp, which):
    """C(t, t') (symmetric) or R(t, t') (0 for t' > t) from the stored history.

    The slice interval containing max(t, t') is found, the theta stencil is placed
    at t_small / t_big on both slices and the result is Hermite-interpolated in t.
    """
    t = np.atleast_1d(np.asarray(t, dtype=float))
    tp = np.atleast_1d(np.asarray(tp, dtype=float))
    t, tp = np.broadcast_arrays(t, tp)
    out = np.zeros(t.shape)
    big = np.maximum(t, tp)
    small = np.minimum(t, tp)
    if np.any(big > hist.t[-1] * (1 + 1e-15)):
        raise ValueError("time beyond the stored history")
    ok = np.ones(t.shape, dtype=bool) if which == "C" else (tp <= t)
    pos = big > 0
    th = np.where(pos, small / np.where(pos, big, 1.0), 1.0)
    om = np.where(pos, (big - small) / np.where(pos, big, 1.0), 0.0)
    x = gridmod.frac_index(th, om, grid.L, grid.gamma, grid.alpha, grid.delta)
    b, w = grid.stencil_at(x, om)
    Y, dY = (hist.C, hist.dC) if which == "C" else (hist.R, hist.dR)
    N = hist.N
    g = lambda rows, m: sum(w[..., k] * rows[m, b + k] for k in range(grid.s))
    positive = lambda m: np.all(np.stack([Y[m, b + k] > 0 for k in range(grid.s)]), axis=0)
    use_log = which == "R" and grid.log_r
    if use_log:
        lY = np.log(np.where(Y > 0, Y, 1.0))
        ldY = dY / np.where(Y > 0, Y, 1.0)
    if N == 1:
        val = g(Y, 0)
        if use_log:
            val = np.where(positive(0), np.exp(g(lY, 0)), val)
    else:
        n = np.clip(np.searchsorted(hist.t, big, side="right") - 1, 0, N - 2)
        h = hist.t[n + 1] - hist.t[n]
        sig = (big - hist.t[n]) / h
        val = hermite(g(Y, n), g(dY, n), g(Y, n + 1), g(dY, n + 1), h, sig)
        if use_log:
            # logarithmic interpolation of the response where the stencil is positive
            lval = np.exp(hermite(g(lY, n), g(ldY, n), g(lY, n + 1), g(ldY, n + 1), h, sig))
            val = np.where(positive(n) & positive(n + 1), lval, val)
    out[ok] = val[ok]
    return out
