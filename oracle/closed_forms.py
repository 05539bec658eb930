"""Independent reference solutions used only to pin the oracle (never the method itself).

1. Pure p = 2 model, f(q) = q^2/2, quench from T = infinity to T = 0 (the paper's
   accuracy test, Sec. 4.2, Fig. 2-accuracy). The couplings have a semicircle
   spectrum on [-2, 2]; each eigenmode relaxes exponentially, which gives with
   g(x) = I_1(2x)/x (the semicircle moment generating function):

       C(t,t') = g(t + t') / sqrt(g(2t) g(2t'))
       R(t,t') = g(t - t') sqrt(g(2t') / g(2t))
       mu(t)   = 2 I_0(4t)/I_1(4t) - 1/t,      E(t) = -mu(t)/2  (E = (T - mu)/2 at T = 0)

   Bessel functions come from scipy.special (exponentially scaled forms).

2. Equilibrium dynamics above T_d (time-translation invariance and FDT,
   R(tau) = -(1/T) dC/dtau): the one-time equation
       C'(tau) = -T C(tau) - (1/T) int_0^tau f'(C(tau - u)) C'(u) du,  C(0) = 1,
   solved on a uniform grid (trapezoid rule, implicit in the newest point) with
   Richardson extrapolation. The energy is -f(1)/T.

3. Brute-force two-time solver on a uniform grid t_a = a h (the O(N^3) baseline
   of Sec. 2.3): explicit Heun in t for C(t_a, t_b), R(t_a, t_b) with trapezoid
   quadrature of all memory integrals, C(t,t) = R(t,t^-) = 1. Second order in h;
   Richardson over h, h/2, h/4 removes the leading error.
"""

import numpy as np
from scipy import special


# ---------------------------------------------------------------- p = 2, T = 0
def _log_g(x):
    """ln g(x), g(x) = I_1(2x)/x (g(0) = 1)."""
    x = np.asarray(x, dtype=float)
    out = np.empty_like(x)
    small = x < 2.0
    xs = x[small]
    ser = np.zeros_like(xs)
    term = np.ones_like(xs)
    for k in range(40):
        ser += term
        term = term * xs * xs / ((k + 1) * (k + 2))
    out[small] = np.log(ser)
    xl = x[~small]
    out[~small] = np.log(special.i1e(2 * xl)) + 2 * xl - np.log(xl)
    return out


def _dlog_g(x):
    """d/dx ln g(x)."""
    x = np.asarray(x, dtype=float)
    out = np.empty_like(x)
    small = x < 2.0
    xs = x[small]
    g = np.zeros_like(xs)
    dg = np.zeros_like(xs)
    term = np.ones_like(xs)  # x^{2k} / (k! (k+1)!)
    for k in range(40):
        g += term
        if k > 0:
            with np.errstate(invalid="ignore", divide="ignore"):
                dg += 2 * k * term / xs
        term = term * xs * xs / ((k + 1) * (k + 2))
    with np.errstate(invalid="ignore", divide="ignore"):
        out[small] = np.where(xs > 0, dg / g, 0.0)
    xl = x[~small]
    out[~small] = 2 * special.i0e(2 * xl) / special.i1e(2 * xl) - 2 / xl
    return out


def p2_C(t, tp):
    t, tp = np.broadcast_arrays(np.asarray(t, float), np.asarray(tp, float))
    return np.exp(_log_g(t + tp) - 0.5 * _log_g(2 * t) - 0.5 * _log_g(2 * tp))


def p2_R(t, tp):
    t, tp = np.broadcast_arrays(np.asarray(t, float), np.asarray(tp, float))
    out = np.exp(_log_g(np.abs(t - tp)) + 0.5 * _log_g(2 * tp) - 0.5 * _log_g(2 * t))
    return np.where(tp <= t, out, 0.0)


def p2_mu(t):
    t = np.asarray(t, dtype=float)
    return _dlog_g(2 * t)  # mu = (1/2) d/dt ln Gamma, Gamma(t) = g(2t)


def p2_E(t):
    return -0.5 * p2_mu(t)


def p2_fields(t, theta, omega):
    """Cf, dCf/dt|theta, Rf, dRf/dt|theta at time t on the theta grid (exact)."""
    t = float(t)
    tp = theta * t
    C = p2_C(t, tp)
    R = p2_R(t, tp)
    # d/dt ln C(t, theta t) = (1+theta) h(t(1+theta)) - h(2t) - theta h(2 theta t)
    dlnC = (1 + theta) * _dlog_g(t * (1 + theta)) - _dlog_g(2 * t) - theta * _dlog_g(2 * theta * t)
    # d/dt ln R(t, theta t) = (1-theta) h(t(1-theta)) + theta h(2 theta t) - h(2t)
    dlnR = omega * _dlog_g(t * omega) + theta * _dlog_g(2 * theta * t) - _dlog_g(2 * t)
    return C, C * dlnC, R, R * dlnR


def p2_history(times, theta, omega):
    """Exact history rows for the stored slice times (times[0] must be 0)."""
    rows = [p2_fields(tt, theta, omega) for tt in times]
    return tuple(np.array([r[k] for r in rows]) for k in range(4))


# ---------------------------------------------------- equilibrium above T_d
def equilibrium_C(fp, T, tau_max, h):
    """C_eq on tau = 0, h, .., tau_max and C_eq' there (second order in h)."""
    n = int(round(tau_max / h))
    beta = 1.0 / T
    C = np.empty(n + 1)
    dC = np.empty(n + 1)
    C[0] = 1.0
    dC[0] = -T
    for k in range(1, n + 1):
        # trapezoid: I_k = h [ f'(C_k) dC_0 / 2 + sum_{m=1}^{k-1} f'(C_{k-m}) dC_m + f'(C_0) dC_k / 2 ]
        c = C[k - 1] + h * dC[k - 1]
        for _ in range(50):
            inner = np.dot(fp(C[k - 1:0:-1]), dC[1:k]) if k > 1 else 0.0
            # dC_k = -T c - beta h [fp(c) dC_0/2 + inner + fp(1) dC_k/2]
            dk = (-T * c - beta * h * (0.5 * fp(c) * dC[0] + inner)) / (1.0 + 0.5 * beta * h * fp(1.0))
            c_new = C[k - 1] + 0.5 * h * (dC[k - 1] + dk)
            if abs(c_new - c) < 1e-15:
                c = c_new
                break
            c = c_new
        C[k] = c
        dC[k] = dk
    return C, dC


def equilibrium_C_richardson(fp, T, tau_max, h):
    """Richardson-extrapolated C_eq, C_eq' on the grid of step h, and an error estimate."""
    C1, d1 = equilibrium_C(fp, T, tau_max, h)
    C2, d2 = equilibrium_C(fp, T, tau_max, h / 2)
    C4, d4 = equilibrium_C(fp, T, tau_max, h / 4)
    Ca = (4 * C2[::2] - C1) / 3
    Cb = (4 * C4[::4] - C2[::2]) / 3
    da = (4 * d2[::2] - d1) / 3
    db = (4 * d4[::4] - d2[::2]) / 3
    return Cb, db, np.max(np.abs(Cb - Ca))


# ------------------------------------------------ brute-force uniform grid
def uniform_solve(model, t_max, h):
    """C[a, b], R[a, b] on t_a = a h for 0 <= b <= a <= N (Heun + trapezoid)."""
    N = int(round(t_max / h))
    T = model.T
    C = np.zeros((N + 1, N + 1))
    R = np.zeros((N + 1, N + 1))
    C[0, 0] = 1.0
    R[0, 0] = 1.0

    def wts(n):
        w = np.full(n + 1, h)
        w[0] = w[-1] = 0.5 * h
        if n == 0:
            w[:] = 0.0
        return w

    def trap(n):
        """Trapezoid weight matrix W[b, s] for the integral over s in [0, t_b]."""
        W = np.zeros((n + 1, n + 1))
        for b in range(n + 1):
            W[b, :b + 1] = wts(b)
        return W

    def derivs(a, Crow, Rrow):
        """d1C(t_a, t_b), d1R(t_a, t_b) for b = 0..a from row a values Crow, Rrow (len a+1)
        and the stored rows b < a (C symmetric, R causal)."""
        w = wts(a)
        K = model.fpp(Crow) * Rrow  # K(a, s) for s = 0..a
        D = model.fp(Crow)
        mu = T + np.dot(w, K * Crow + D * Rrow)
        # C(s, b) for s, b in 0..a: symmetric matrix from stored rows and row a
        Cm = C[:a + 1, :a + 1].copy()
        Cm[a, :a + 1] = Crow
        Cm = np.tril(Cm) + np.tril(Cm, -1).T
        Rm = R[:a + 1, :a + 1].copy()  # Rm[b, s] = R(t_b, t_s), zero for s > b
        Rm[a, :a + 1] = Rrow
        Rm = np.tril(Rm)
        Wlow = trap(a)                     # Wlow[b, s]: trapezoid on [0, t_b]
        Wup = np.zeros((a + 1, a + 1))     # Wup[b, s]: trapezoid on [t_b, t_a]
        for b in range(a + 1):
            Wup[b, b:] = wts(a - b)
        i1 = (w * K) @ Cm                  # int_0^{t_a} K(a,s) C(s,b) ds
        i2 = (Wlow * Rm) @ D               # int_0^{t_b} D(a,s) R(b,s) ds
        i3 = (Wup * Rm.T) @ K              # int_{t_b}^{t_a} K(a,s) R(s,b) ds
        return -mu * Crow + i1 + i2, -mu * Rrow + i3

    for a in range(N):
        Ca, Ra = C[a, :a + 1].copy(), R[a, :a + 1].copy()
        dC0, dR0 = derivs(a, Ca, Ra)
        Cp = np.append(Ca + h * dC0, 1.0)
        Rp = np.append(Ra + h * dR0, 1.0)
        dC1, dR1 = derivs(a + 1, Cp, Rp)
        C[a + 1, :a + 1] = Ca + 0.5 * h * (dC0 + dC1[:a + 1])
        R[a + 1, :a + 1] = Ra + 0.5 * h * (dR0 + dR1[:a + 1])
        C[a + 1, a + 1] = 1.0
        R[a + 1, a + 1] = 1.0
    return C, R
