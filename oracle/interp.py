"""Interpolation of Sec. 3.3: index-space Lagrange stencils and cubic Hermite in t.

Lagrange (the paper's default "index interpolation"): the field is interpolated
in the 0-based index x of the theta grid, on which it is smooth. An s-point
stencil starts at b = clamp(floor(x) - s/2 + 1, 0, L - s) (one-sided at the two
ends; reading of the stencil placement) and uses the Lagrange basis on the
equispaced nodes 0..s-1 evaluated at u = x - b.

Hermite: between stored slices t_n < t_{n+1} with values y and stored time
derivatives y', the local cubic Hermite interpolant (Sec. 3.3, the "local cubic
Hermite interpolation on the adaptive grid in t").

Pins: tests/test_oracle_interp.py (polynomial reproduction of degree s-1,
convergence order, Hermite reproduction of cubics).
"""

import numpy as np


def lagrange_stencil(x, L, s):
    """Return (b, w): integer base index and the s Lagrange weights at x.

    x may be an array of any shape; b has that shape and w one more axis of
    length s, so that value = sum_k w[..., k] * row[b + k].
    """
    x = np.asarray(x, dtype=float)
    b = np.clip(np.floor(x).astype(np.int64) - s // 2 + 1, 0, L - s)
    u = x - b
    w = np.ones(x.shape + (s,))
    for k in range(s):
        for m in range(s):
            if m != k:
                w[..., k] *= (u - m) / (k - m)
    return b, w


def apply_stencil(row_of, b, w):
    """sum_k w[..., k] * row_of(b + k) for a callable giving gathered values."""
    s = w.shape[-1]
    out = 0.0
    for k in range(s):
        out = out + w[..., k] * row_of(b + k)
    return out


def hermite_basis(sig):
    """Cubic Hermite basis (h00, h10, h01, h11) at the fraction sig of the interval."""
    sig = np.asarray(sig, dtype=float)
    om = 1.0 - sig
    h00 = (1.0 + 2.0 * sig) * om * om
    h10 = sig * om * om
    h01 = sig * sig * (3.0 - 2.0 * sig)
    h11 = sig * sig * (sig - 1.0)
    return h00, h10, h01, h11


def hermite(y0, d0, y1, d1, h, sig):
    """Cubic Hermite value at t_n + sig*h from (y, y') at both ends of [t_n, t_n + h]."""
    h00, h10, h01, h11 = hermite_basis(sig)
    return h00 * y0 + h10 * h * d0 + h01 * y1 + h11 * h * d1


def hermite_integral(y0, d0, y1, d1, h):
    """Exact integral of the cubic Hermite interpolant over an interval of length h."""
    return 0.5 * h * (y0 + y1) + h * h * (d0 - d1) / 12.0
