"""Pins for oracle/interp.py (Sec. 3.3)."""
import numpy as np
import pytest

from oracle.interp import lagrange_stencil, hermite, hermite_integral


@pytest.mark.parametrize("s", [2, 4, 6, 10])
def test_lagrange_reproduces_polynomials_of_degree_below_s(s):
    L = 40
    rng = np.random.default_rng(1)
    coef = rng.normal(size=s)
    row = np.polyval(coef, np.arange(L, dtype=float))
    x = np.concatenate([rng.uniform(0, L - 1, 200), [0.0, L - 1.0, 0.5, L - 1.5]])
    b, w = lagrange_stencil(x, L, s)
    assert np.all(b >= 0) and np.all(b + s <= L)
    val = sum(w[:, k] * row[b + k] for k in range(s))
    exact = np.polyval(coef, x)
    assert np.max(np.abs(val - exact)) < 1e-8 * np.max(np.abs(row))


@pytest.mark.parametrize("s", [4, 6])
def test_lagrange_converges_at_order_s(s):
    errs = []
    for L in [33, 65, 129]:
        xs = np.linspace(0.0, 1.0, L)
        row = np.sin(3 * xs) + xs ** 7
        xq = np.linspace(0.0, L - 1.0, 997)
        b, w = lagrange_stencil(xq, L, s)
        val = sum(w[:, k] * row[b + k] for k in range(s))
        t = xq / (L - 1)
        errs.append(np.max(np.abs(val - (np.sin(3 * t) + t ** 7))))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > s - 0.6)


def test_stencil_placement_is_centred_and_one_sided_at_the_ends():
    b, _ = lagrange_stencil(np.array([0.2, 5.5, 38.9]), 40, 4)
    assert list(b) == [0, 4, 36]
    b, _ = lagrange_stencil(np.array([5.5]), 40, 10)
    assert list(b) == [1]


def test_hermite_reproduces_cubics_and_its_integral_is_exact():
    rng = np.random.default_rng(2)
    c = rng.normal(size=4)
    p = np.poly1d(c)
    dp = p.deriv()
    a, h = 0.7, 0.3
    sig = np.linspace(0, 1, 11)
    val = hermite(p(a), dp(a), p(a + h), dp(a + h), h, sig)
    assert np.max(np.abs(val - p(a + sig * h))) < 1e-13
    P = p.integ()
    assert abs(hermite_integral(p(a), dp(a), p(a + h), dp(a + h), h) - (P(a + h) - P(a))) < 1e-14


# ---- Floater-Hormann and theta-space stencils (the other options of Sec. 3.3)
from oracle.interp import fh_weights, scheme_stencil  # noqa: E402


@pytest.mark.parametrize("s", [4, 6, 10])
def test_fh_with_full_degree_is_the_lagrange_stencil(s):
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 39, 300)
    b, wl = lagrange_stencil(x, 40, s)
    b2, wf = scheme_stencil(x, None, None, 40, s, "fh_index", s - 1)
    assert np.array_equal(b, b2)
    assert np.max(np.abs(wf - wl)) < 1e-12


def test_fh_degree_zero_is_berrut():
    # d = 0: beta_k = (-1)^k (Berrut 1988), r(x) = sum (-1)^k f_k/(x-x_k) / sum (-1)^k/(x-x_k)
    nodes = np.array([0.0, 0.7, 1.1, 2.5, 3.0])
    x = 1.9
    q = np.array([(-1.0) ** k / (x - nodes[k]) for k in range(5)])
    assert np.max(np.abs(fh_weights(nodes, np.array(x), 0) - q / q.sum())) < 1e-15


@pytest.mark.parametrize("s,d", [(6, 2), (8, 3), (10, 3), (10, 5)])
def test_fh_reproduces_degree_d_and_sums_to_one(s, d):
    rng = np.random.default_rng(4)
    coef = rng.normal(size=d + 1)
    row = np.polyval(coef, np.arange(40, dtype=float))
    x = np.concatenate([rng.uniform(0, 39, 200), [0.0, 3.0, 39.0]])
    b, w = scheme_stencil(x, None, None, 40, s, "fh_index", d)
    val = sum(w[:, k] * row[b + k] for k in range(s))
    assert np.max(np.abs(val - np.polyval(coef, x))) < 1e-9 * np.max(np.abs(row))
    assert np.max(np.abs(w.sum(axis=1) - 1.0)) < 1e-13
    # a point on a node returns that node's value
    assert np.max(np.abs(val[-3:] - row[[0, 3, 39]])) < 1e-12 * np.max(np.abs(row))


def test_fh_converges_at_order_d_plus_one():
    s, d = 8, 3
    errs = []
    for L in [65, 129, 257]:
        xs = np.linspace(0.0, 1.0, L)
        row = np.sin(3 * xs) + xs ** 7
        xq = np.linspace(0.0, L - 1.0, 1999)
        b, w = scheme_stencil(xq, None, None, L, s, "fh_index", d)
        val = sum(w[:, k] * row[b + k] for k in range(s))
        t = xq / (L - 1)
        errs.append(np.max(np.abs(val - (np.sin(3 * t) + t ** 7))))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > d + 1 - 0.5), rates


@pytest.mark.parametrize("scheme", ["lagrange_theta", "fh_theta"])
def test_theta_space_schemes_reproduce_polynomials_in_theta(scheme):
    from oracle.grid import gamma_from_tmax, theta_grid, frac_index
    L, s = 65, 6
    g = gamma_from_tmax(100.0)
    th, om = theta_grid(L, g, 0.0, 0.0)
    d = s - 1 if scheme == "lagrange_theta" else 2
    coef = np.random.default_rng(5).normal(size=d + 1)
    row = np.polyval(coef, om)                      # a polynomial in 1 - theta
    omq = np.linspace(1e-6, 1.0, 400)
    x = frac_index(1.0 - omq, omq, L, g, 0.0, 0.0)
    b, w = scheme_stencil(x, omq, om, L, s, scheme, d)
    val = sum(w[:, k] * row[b + k] for k in range(s))
    assert np.max(np.abs(val - np.polyval(coef, omq))) < 1e-10
