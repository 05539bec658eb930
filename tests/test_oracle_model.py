"""Pins for oracle/model.py (Sec. 2.1)."""
import numpy as np

from oracle.model import Model


def test_derivatives_against_finite_differences():
    m = Model({3: 0.25, 4: 0.25, 2: 0.1}, T=0.5)
    q = np.linspace(-0.9, 0.95, 23)
    h = 1e-5
    assert np.max(np.abs(m.fp(q) - (m.f(q + h) - m.f(q - h)) / (2 * h))) < 1e-9
    assert np.max(np.abs(m.fpp(q) - (m.fp(q + h) - m.fp(q - h)) / (2 * h))) < 1e-9


def test_pure_three_spin_closed_forms():
    m = Model({3: 0.5}, T=0.8)
    q = np.array([0.0, 0.3, 1.0])
    assert np.allclose(m.f(q), 0.5 * q ** 3)
    assert np.allclose(m.fp(q), 1.5 * q ** 2)
    assert np.allclose(m.fpp(q), 3.0 * q)
