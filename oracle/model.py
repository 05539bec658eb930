"""The spherical mixed p-spin model of Sec. 2.1.

Covariance f(q) = sum_p c_p q^p (the paper writes sum alpha_p^2/2 q^p and, for two
terms, lambda q^p + (1 - lambda) q^s; here the coefficients are an arbitrary
input, which covers both normalisations). Memory kernels K = f''(C) R,
D = f'(C); forcing F_C = beta0 f'(C(t,0)) C(t',0); bath temperature T.

Pins: tests/test_oracle_model.py (derivatives against finite differences of f).
"""

import numpy as np


class Model:
    def __init__(self, coefs, T, beta0=0.0):
        """coefs: mapping power p (int >= 1) -> coefficient c_p."""
        self.terms = sorted((int(p), float(c)) for p, c in dict(coefs).items())
        if any(p < 1 for p, _ in self.terms):
            raise ValueError("powers must be >= 1")
        self.T = float(T)
        self.beta0 = float(beta0)

    def f(self, q):
        q = np.asarray(q, dtype=float)
        return sum(c * q ** p for p, c in self.terms) + 0.0 * q

    def fp(self, q):
        """f'(q)."""
        q = np.asarray(q, dtype=float)
        return sum(c * p * q ** (p - 1) for p, c in self.terms) + 0.0 * q

    def fpp(self, q):
        """f''(q)."""
        q = np.asarray(q, dtype=float)
        return sum(c * p * (p - 1) * q ** (p - 2) for p, c in self.terms if p >= 2) + 0.0 * q
