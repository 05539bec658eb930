"""Pins for oracle/integrals.py (Secs. 2.1, 3.3, 3.4)."""
import numpy as np
import pytest
from scipy.integrate import quad

from oracle import closed_forms as cf
from oracle import integrals as I
from oracle.model import Model
from oracle.integrals import Grid, History

P2 = Model({2: 0.5}, T=0.0)  # f(q) = q^2/2: f' = q, f'' = 1


def _p2_history(G, t_last, n, t_first=1e-3):
    times = np.concatenate([[0.0], np.geomspace(t_first, t_last, n)])
    return History(times, *cf.p2_history(times, G.theta, G.omega))


def _exact_rows(t, thj):
    """Exact integrands of S[0..8] at output theta_j for f = q^2/2 (functions of theta_i)."""
    C, R = cf.p2_C, cf.p2_R
    tp = thj * t
    p1 = lambda x: x * thj
    p2 = lambda x: thj + (1 - thj) * x
    return [
        lambda x: R(t, p1(x) * t) * C(tp, p1(x) * t),
        lambda x: R(t, p2(x) * t) * C(p2(x) * t, tp),
        lambda x: C(t, p1(x) * t) * R(tp, p1(x) * t),
        lambda x: R(t, p2(x) * t) * R(p2(x) * t, tp),
        lambda x: R(tp, p1(x) * t) * C(t, p1(x) * t),
        lambda x: C(tp, p1(x) * t) * R(t, p1(x) * t),
        lambda x: C(p2(x) * t, tp) * R(t, p2(x) * t),
        lambda x: R(p2(x) * t, tp) * R(t, p2(x) * t),
        lambda x: 2 * C(tp, p1(x) * t) * R(tp, p1(x) * t),
    ]


def test_each_sum_against_adaptive_quadrature_of_exact_p2_integrand():
    """S[r][j] = int_0^1 (integrand r) dtheta_i, pinned row by row by scipy quad."""
    G = Grid(257, 100.0, s=6)
    t = 4.0
    H = _p2_history(G, t, 1200)
    C, R = H.C[-1], H.R[-1]
    S = I.history_integrals(P2, G, H, t, C, R)
    for j in [0, 40, 128, 200, 250, 256]:
        rows = _exact_rows(t, G.theta[j])
        for r, fn in enumerate(rows):
            ref, _ = quad(lambda x: float(fn(np.array([x]))[0]), 0.0, 1.0, epsabs=1e-13, epsrel=1e-12, limit=200)
            assert abs(S[r, j] - ref) < 2e-7, (r, j, S[r, j], ref)
    # S[9] = C(theta_j t, 0)
    assert np.max(np.abs(S[9] - cf.p2_C(G.theta * t, 0.0))) < 1e-7


def test_rhs_matches_exact_p2_derivative_and_converges_in_L():
    errs = []
    for L in [65, 129]:
        G = Grid(L, 100.0, s=4)
        t = 5.0
        H = _p2_history(G, t, 400)
        dC, dR, mu, E = I.rhs(P2, G, H, t, H.C[-1], H.R[-1])
        _, dCx, _, dRx = cf.p2_fields(t, G.theta, G.omega)
        errs.append(max(np.max(np.abs(dC - dCx)), np.max(np.abs(dR - dRx))))
        assert abs(mu - cf.p2_mu(t)) < 1e-6 and abs(E - cf.p2_E(t)) < 1e-6
    assert errs[1] < errs[0] / 8
    assert errs[1] < 2e-6


def test_rhs_converges_with_stencil_width():
    G = Grid(129, 100.0, s=6)
    t = 5.0
    H = _p2_history(G, t, 400)
    dC, dR, _, _ = I.rhs(P2, G, H, t, H.C[-1], H.R[-1])
    _, dCx, _, dRx = cf.p2_fields(t, G.theta, G.omega)
    assert max(np.max(np.abs(dC - dCx)), np.max(np.abs(dR - dRx))) < 5e-8


def test_free_model_is_exact():
    """f = 0: C(t,t') = R(t,t') = exp(-T (t - t')), so dCf/dt|theta = -T (1 - theta) Cf."""
    T = 0.7
    m = Model({2: 0.0}, T=T)
    G = Grid(65, 100.0)
    times = np.array([0.0, 0.5, 1.0, 1.7])
    ex = lambda tt: np.exp(-T * tt * G.omega)
    rows = [ex(tt) for tt in times]
    drows = [-T * G.omega * r for r in rows]
    H = History(times, rows, drows, rows, drows)
    dC, dR, mu, E = I.rhs(m, G, H, 1.7, rows[-1], rows[-1])
    assert np.max(np.abs(dC - drows[-1])) < 1e-14 and np.max(np.abs(dR - drows[-1])) < 1e-14
    assert mu == T and E == 0.0


def _smooth_history(G, seed=3):
    rng = np.random.default_rng(seed)
    times = np.concatenate([[0.0], np.geomspace(0.01, 3.0, 60)])
    a, b = rng.uniform(0.3, 0.8, 2)
    C = np.array([np.exp(-a * tt * G.omega) * (1 + 0.1 * np.sin(tt * G.theta)) for tt in times])
    C[:, -1] = 1.0
    R = np.array([np.exp(-b * tt * G.omega) for tt in times])
    dC = np.gradient(C, times, axis=0)
    dR = np.gradient(R, times, axis=0)
    return History(times, C, dC, R, dR)


def test_pure_model_mu_equals_T_minus_pE():
    """For f = c q^p, f''(q) q = (p-1) f'(q), so mu - T = -p E holds term by term."""
    m = Model({3: 0.5}, T=0.8)
    G = Grid(65, 100.0)
    H = _smooth_history(G)
    _, _, mu, E = I.row_prep(m, G, 3.0, H.C[-1], H.R[-1])
    assert abs(mu - (0.8 - 3 * E)) < 1e-13


def test_diagonal_derivatives_vanish_before_pinning():
    """At theta = 1: d1C = -T, d2C = +T, d1R = -mu, d2R = +mu (C(t,t) = 1, R(t,t^-) = 1)."""
    m = Model({3: 0.25, 4: 0.25}, T=0.5)
    G = Grid(65, 100.0)
    H = _smooth_history(G)
    t = H.t[-1]
    C, R = H.C[-1], H.R[-1]
    _, _, mu, _ = I.row_prep(m, G, t, C, R)
    S = I.history_integrals(m, G, H, t, C, R)
    j = G.L - 1
    d1C = -mu + t * (S[0, j] + S[2, j])
    mu_p = m.T + t * S[8, j]
    d2C = -mu_p + t * (S[4, j] + S[5, j]) + 2 * m.T
    assert abs(d1C + m.T) < 1e-11
    assert abs(mu_p - mu) < 1e-11
    assert abs(d2C - m.T) < 1e-11


@pytest.mark.parametrize("mutation", ["swap_S0_S1", "drop_d2", "psi_numerator"])
def test_planted_mistakes_are_caught_by_the_p2_pin(mutation):
    """A plausible slip in the oracle (wrong row, dropped term, swapped operand) fails P1."""
    G = Grid(129, 100.0, s=6)
    t = 5.0
    H = _p2_history(G, t, 400)
    C, R = H.C[-1], H.R[-1]
    _, _, mu, _ = I.row_prep(P2, G, t, C, R)
    S = I.history_integrals(P2, G, H, t, C, R)
    if mutation == "swap_S0_S1":
        S = S[[1, 0, 2, 3, 4, 5, 6, 7, 8, 9]]
        dC, dR = I.assemble_rhs(P2, G, t, C, R, S, mu)
    elif mutation == "drop_d2":
        d1C = -mu * C + t * (G.theta * (S[0] + S[2]) + G.omega * S[1])
        dC, dR = d1C, -mu * R + t * G.omega * S[3]
    else:  # B2 read at theta_i / phi2 instead of theta_j / phi2 (phi2 itself is symmetric)
        G2 = Grid(129, 100.0, s=6)
        phi2, x1, x2, x3, o1, o2, o3 = G2._cache
        G2._cache = (phi2, x1, x2, x3.T.copy(), o1, o2, o3.T.copy())
        S = I.history_integrals(P2, G2, H, t, C, R)
        dC, dR = I.assemble_rhs(P2, G, t, C, R, S, mu)
    _, dCx, _, dRx = cf.p2_fields(t, G.theta, G.omega)
    err = max(np.max(np.abs(dC[:-1] - dCx[:-1])), np.max(np.abs(dR[:-1] - dRx[:-1])))
    assert err > 1e-3


# ---- logarithmic interpolation of the response history (App. A)
def _exp_history(L, s, sign_flip=False):
    """R(t_n, x) = exp(a + b x + c t_n) on the grid index x: log R is linear in t and in x,
    so the logarithmic interpolation reproduces it exactly and the linear one does not."""
    G = Grid(L, 100.0, s=s, log_r=True)
    t = np.array([0.0, 0.5, 1.1, 1.8, 2.6])
    x = np.arange(L, dtype=float)
    a, bb, c = -0.3, -0.05, -0.7
    R = np.exp(a + bb * x[None, :] + c * t[:, None])
    dR = c * R
    C = 0.5 * R
    if sign_flip:
        R[2, 10:14] *= -1.0
        dR[2, 10:14] *= -1.0
    return G, History(t, C, 0.5 * dR, R, dR), (a, bb, c)


def test_log_r_reproduces_exponential_response():
    from oracle.integrals import lookup
    L, s = 65, 6
    G, H, (a, bb, c) = _exp_history(L, s)
    rng = np.random.default_rng(8)
    xq = rng.uniform(0, L - 1, 300)
    tq = rng.uniform(0.0, 2.6, 300)
    b, w = G.stencil_at(xq, None)
    _, R_log = lookup(H, tq, b, w, 2.6, H.C[-1], H.R[-1], log_r=True)
    _, R_lin = lookup(H, tq, b, w, 2.6, H.C[-1], H.R[-1], log_r=False)
    exact = np.exp(a + bb * xq + c * tq)
    assert np.max(np.abs(R_log - exact) / exact) < 1e-12
    assert np.max(np.abs(R_lin - exact) / exact) > 1e-6      # the linear path is only approximate
    # beyond the last slice: the quadratic extension in log R, exact for log R linear in t
    t_cur = 3.0
    row = np.exp(a + bb * np.arange(L) + c * t_cur)
    tq2 = rng.uniform(2.6, 3.0, 100)
    xq2 = rng.uniform(0, L - 1, 100)
    b2, w2 = G.stencil_at(xq2, None)
    _, R2 = lookup(H, tq2, b2, w2, t_cur, 0.5 * row, row, log_r=True)
    assert np.max(np.abs(R2 - np.exp(a + bb * xq2 + c * tq2)) / R2) < 1e-12


def test_log_r_falls_back_where_the_stencil_is_not_positive():
    from oracle.integrals import lookup
    L, s = 65, 4
    G, H, _ = _exp_history(L, s, sign_flip=True)
    xq = np.array([11.3, 40.2, 12.0])
    tq = np.array([1.4, 1.4, 0.8])       # all in the intervals that touch slice 2 (t = 1.1)
    b, w = G.stencil_at(xq, None)
    _, R_log = lookup(H, tq, b, w, 2.6, H.C[-1], H.R[-1], log_r=True)
    _, R_lin = lookup(H, tq, b, w, 2.6, H.C[-1], H.R[-1], log_r=False)
    assert R_log[0] == R_lin[0] and R_log[2] == R_lin[2]     # stencils touching the negative values
    assert R_log[1] != R_lin[1]                               # a positive stencil takes the log path


def test_log_r_two_time_lookup():
    from oracle import grid as gm
    from oracle.solver import get_two_time
    L, s = 65, 6
    G, H, (a, bb, c) = _exp_history(L, s)
    t = np.array([2.6, 2.0, 1.3, 0.7])
    tp = np.array([1.0, 0.3, 1.2, 0.1])
    th, om = tp / t, (t - tp) / t
    x = gm.frac_index(th, om, L, G.gamma, G.alpha, G.delta)
    got = get_two_time(G, H, t, tp, "R")
    assert np.max(np.abs(got - np.exp(a + bb * x + c * t)) / got) < 1e-12


def test_log_r_solve_converges_to_the_linear_solve():
    """Both readings of the response interpolation discretise the same equations: the
    difference between a solve with log-R interpolation and the default solve is
    discretisation error, which falls fast with L (~85x from L = 17 to 33 at s = 6), while
    the equal-time values stay exact."""
    from oracle import solver as S
    t = np.array([1.0, 1.0, 0.75, 0.4])
    tp = np.array([0.0, 0.5, 0.7, 0.2])
    diff = {}
    for L in (17, 33):
        kw = dict(L=L, grid_t_max=100.0, s=6, history_cap=60)
        a = S.Solver({3: 0.25, 4: 0.25}, 0.5, log_r=True, **kw)
        b = S.Solver({3: 0.25, 4: 0.25}, 0.5, **kw)
        assert a.integrate(1.0, 1e-9) == S.OK and b.integrate(1.0, 1e-9) == S.OK
        diff[L] = (np.max(np.abs(a.get_R(t, tp) - b.get_R(t, tp))), abs(a.E - b.E))
        ts = np.array([0.5, 1.0])
        assert np.max(np.abs(a.get_R(ts, ts) - 1.0)) < 1e-14
    assert 0.0 < diff[33][0] < diff[17][0] / 16 and diff[33][0] < 1e-5
    assert diff[33][1] < diff[17][1] / 16
