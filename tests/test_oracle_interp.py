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
