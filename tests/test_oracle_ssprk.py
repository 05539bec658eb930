"""Pins for the SSPRK(10,4) integrator and the Dormand-Prince -> SSPRK switch of the
oracle (Sec. 3.5): order conditions, the low-storage recurrence, convergence orders,
stability polynomials and the switch rule inside a solve."""
from fractions import Fraction as Fr

import numpy as np
import pytest

from oracle import solver as S


def _elementary(c, A, b):
    """The eight Butcher order conditions up to order 4 (rooted trees), exact."""
    n = len(b)
    Ac = [sum(A[i][l] * c[l] for l in range(i)) for i in range(n)]
    Ac2 = [sum(A[i][l] * c[l] ** 2 for l in range(i)) for i in range(n)]
    AAc = [sum(A[i][l] * Ac[l] for l in range(i)) for i in range(n)]
    s = lambda v: sum(bi * vi for bi, vi in zip(b, v))
    return [s([1] * n), s(c), s([x * x for x in c]), s(Ac),
            s([x ** 3 for x in c]), s([ci * a for ci, a in zip(c, Ac)]), s(Ac2), s(AAc)]


TARGETS = [Fr(1), Fr(1, 2), Fr(1, 3), Fr(1, 6), Fr(1, 4), Fr(1, 8), Fr(1, 12), Fr(1, 24)]


def test_ssprk104_tableau_order_conditions():
    c, A, b, bhat = S.ssprk104_exact()
    assert len(c) == 10 and all(len(A[i]) == i for i in range(10))
    # Ketcheson's method: uniform weights 1/10, abscissae 0,1/6,..,2/3, 1/3,..,1
    assert b == [Fr(1, 10)] * 10
    assert c == [Fr(k, 6) for k in range(5)] + [Fr(1, 3), Fr(1, 2), Fr(2, 3), Fr(5, 6), Fr(1)]
    assert _elementary(c, A, b) == TARGETS                  # order 4
    eh = _elementary(c, A, bhat)
    assert eh[:4] == TARGETS[:4]                             # embedded: order 3 ...
    assert eh[4] != TARGETS[4]                               # ... and not 4
    assert bhat[9] == 0 and min(bhat) >= 0
    # minimal 2-norm among order-3 vectors with zero last weight: bhat is in the span of
    # the condition rows (1, c, c^2, A c) restricted to the first nine stages
    Ac = [sum(A[i][l] * c[l] for l in range(i)) for i in range(10)]
    M = np.array([[1.0] * 9, [float(x) for x in c[:9]], [float(x) ** 2 for x in c[:9]],
                  [float(x) for x in Ac[:9]]]).T
    coef, res, *_ = np.linalg.lstsq(M, np.array([float(x) for x in bhat[:9]]), rcond=None)
    assert np.max(np.abs(M @ coef - np.array([float(x) for x in bhat[:9]]))) < 1e-14


def test_ssprk104_reproduces_low_storage_recurrence():
    """The Butcher form against the register recurrence, on a nonlinear autonomous ODE."""
    f = lambda t, y: np.cos(y) - 0.3 * y ** 3
    y0, h = np.array([0.7, -1.1]), 0.37
    q1, q2 = y0.copy(), y0.copy()
    for _ in range(5):
        q1 = q1 + h / 6 * f(0, q1)
    q2 = q2 / 25 + 9 * q1 / 25
    q1 = 15 * q2 - 5 * q1
    for _ in range(4):
        q1 = q1 + h / 6 * f(0, q1)
    ref = q2 + 3 * q1 / 5 + h / 10 * f(0, q1)
    got, _, ks = S.rk_step(S.SSPRK104, f, 0.0, y0, h, f(0, y0))
    assert np.max(np.abs(got - ref)) < 1e-14
    assert np.max(np.abs(ks[-1] - f(0, got))) < 1e-15        # first-same-as-last stage


def test_ssprk104_orders_on_scalar_ode():
    f = lambda t, y: np.array([-y[0] + np.sin(3 * t)])
    exact = lambda t: (np.exp(-t) * (1 + 3 / 10) + (np.sin(3 * t) - 3 * np.cos(3 * t)) / 10)
    errs, ests = [], []
    hs = [0.4, 0.2, 0.1, 0.05]
    for h in hs:
        y0 = np.array([exact(0.3)])
        y1, est, _ = S.rk_step(S.SSPRK104, f, 0.3, y0, h, f(0.3, y0))
        errs.append(abs(y1[0] - exact(0.3 + h)))
        ests.append(abs(est[0]))
    slope = lambda e: np.polyfit(np.log(hs), np.log(e), 1)[0]
    assert slope(errs) > 4.6           # local error of the 4th-order solution, O(h^5)
    assert 3.6 < slope(ests) < 4.5     # third-order embedded estimate, O(h^4)


def test_stability_polynomials_and_dp5_interval():
    g = S.stability_coefficients(S.DP5)
    # DP5: exp(z) to order 5, sixth coefficient 1/600 (Hairer, Norsett & Wanner)
    assert np.allclose(g, [1, 1, 1 / 2, 1 / 6, 1 / 24, 1 / 120, 1 / 600], rtol=1e-13, atol=0)
    gs = S.stability_coefficients(S.SSPRK104)
    assert np.allclose(gs[:5], [1, 1, 1 / 2, 1 / 6, 1 / 24], rtol=1e-13, atol=0)
    # the real interval by direct amplification of one step of y' = lam y
    lin = lambda x, m: abs(S.rk_step(m, lambda t, y: -x * y, 0.0, np.array([1.0]), 1.0,
                                     np.array([-x]))[0][0])
    b = S.DP5_REAL_STABILITY
    assert 3.2 < b < 3.4
    assert lin(b - 1e-6, S.DP5) <= 1.0 < lin(b + 1e-6, S.DP5)
    assert all(lin(x, S.DP5) <= 1.0 for x in np.linspace(0.01, b - 1e-6, 200))
    bs = S.real_stability_boundary(S.SSPRK104)
    # SSP coefficient 6: the disc |z + 6| <= 6 is stable, so the interval covers [-12, 0]
    assert bs > 12.0
    assert lin(bs - 1e-6, S.SSPRK104) <= 1.0 < lin(bs + 1e-6, S.SSPRK104)


def test_switch_dt_auto():
    from oracle.model import Model
    m = Model({3: 0.25, 4: 0.25}, 0.5)       # f''(1) = 1.5 + 3 = 4.5
    assert abs(S.switch_dt_auto(m) - S.DP5_REAL_STABILITY / (4 * np.sqrt(4.5))) < 1e-15
    assert 0.38 < S.switch_dt_auto(m) < 0.40
    assert S.switch_dt_auto(Model({1: 0.5}, 0.5)) == np.inf   # f'' = 0: no stiffness bound


@pytest.fixture(scope="module")
def switch_runs():
    kw = dict(L=33, grid_t_max=100.0, history_cap=400)
    a = S.Solver({3: 0.5}, 0.8, integrator="auto", switch_dt=0.02, **kw)
    assert a.integrate(3.0, 1e-9) == S.OK
    d = S.Solver({3: 0.5}, 0.8, integrator="dp5", **kw)
    assert d.integrate(3.0, 1e-9) == S.OK
    return a, d


def test_switch_happens_once_with_halved_step(switch_runs):
    a, _ = switch_runs
    assert a.method is S.SSPRK104 and a.t_switch is not None
    steps = [e for e in a.log if e[3]]
    k = next(i for i, e in enumerate(steps) if e[0] >= a.t_switch - 1e-15)
    # the step taken right after the switch is about half the last DP5 step
    last_dp, first_ssp = steps[k - 1][1], steps[k][1]
    assert abs(first_ssp / last_dp - 0.5) < 0.02
    assert last_dp * 1.01 >= 0.02 * 0.999


def test_switched_solution_agrees_with_dp5(switch_runs):
    a, d = switch_runs
    t = np.array([3.0, 3.0, 2.5, 1.0])
    tp = np.array([1.0, 0.0, 2.0, 0.5])
    # both runs are within a few tolerances of the true solution at tol 1e-9 over L = 33
    assert np.max(np.abs(a.get_C(t, tp) - d.get_C(t, tp))) < 1e-6
    assert np.max(np.abs(a.get_R(t, tp) - d.get_R(t, tp))) < 1e-6
    assert abs(a.E - d.E) < 1e-6
