"""Interpolation of Sec. 3.3: theta stencils and cubic Hermite in t.

Lagrange (the paper's default "index interpolation"): the field is interpolated
in the 0-based index x of the theta grid, on which it is smooth. An s-point
stencil starts at b = clamp(floor(x) - s/2 + 1, 0, L - s) (one-sided at the two
ends; reading of the stencil placement) and uses the Lagrange basis on the
equispaced nodes 0..s-1 evaluated at u = x - b.

The other options of Sec. 3.3 on the same stencil: Floater-Hormann rational
interpolation (Floater & Hormann 2007) with blending degree d, and both schemes on the
theta values of the stencil nodes instead of their indices. In theta space the nodes
and the point are taken as complements 1 - theta (the grid accumulates at theta = 1,
where differences of theta itself lose their digits); both interpolants are invariant
under that affine change. Floater-Hormann with d = s - 1 is the polynomial interpolant.

Hermite: between stored slices t_n < t_{n+1} with values y and stored time
derivatives y', the local cubic Hermite interpolant (Sec. 3.3, the "local cubic
Hermite interpolation on the adaptive grid in t").

Pins: tests/test_oracle_interp.py (polynomial reproduction of degree s-1,
convergence order, Hermite reproduction of cubics; Floater-Hormann: d = s-1 equals the
Lagrange stencil, d = 0 is Berrut's interpolant with weights (-1)^k, reproduction of
degree-d polynomials, partition of unity, convergence order d + 1; theta-space Lagrange
reproduces polynomials in theta).
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


def fh_weights(nodes, pt, d):
    """Floater-Hormann interpolation weights at pt on the given nodes (last axis, size s).

    Barycentric weights beta_k = sum over i in J_k of (-1)^i prod_{j=i..i+d, j != k}
    1/(x_k - x_j), J_k = {i : max(0, k-d) <= i <= min(k, s-1-d)}; the interpolant is
    sum_k beta_k/(x - x_k) f_k / sum_k beta_k/(x - x_k), and a point on a node takes that
    node's value.
    """
    nodes = np.asarray(nodes, dtype=float)
    pt = np.asarray(pt, dtype=float)
    s = nodes.shape[-1]
    if not 0 <= d <= s - 1:
        raise ValueError("blending degree must be in 0 .. s-1")
    beta = np.zeros(nodes.shape)
    for k in range(s):
        for i in range(max(0, k - d), min(k, s - 1 - d) + 1):
            term = np.full(nodes.shape[:-1], (-1.0) ** i)
            for j in range(i, i + d + 1):
                if j != k:
                    term = term / (nodes[..., k] - nodes[..., j])
            beta[..., k] += term
    diff = pt[..., None] - nodes
    on_node = diff == 0.0
    safe = np.where(on_node, 1.0, diff)
    q = beta / safe
    w = q / np.sum(q, axis=-1, keepdims=True)
    hit = np.any(on_node, axis=-1)
    if np.any(hit):
        w[hit] = on_node[hit].astype(float)
    return w


SCHEMES = ("lagrange_index", "fh_index", "lagrange_theta", "fh_theta")


def scheme_stencil(x, om_pt, omega, L, s, scheme="lagrange_index", d=3):
    """(b, w) of the theta stencil at fractional index x for a scheme of Sec. 3.3.

    om_pt is 1 - theta of the point and omega the grid's complements (theta schemes).
    """
    if scheme == "lagrange_index":
        return lagrange_stencil(x, L, s)
    x = np.asarray(x, dtype=float)
    b = np.clip(np.floor(x).astype(np.int64) - s // 2 + 1, 0, L - s)
    dd = s - 1 if scheme.startswith("lagrange") else d
    if scheme.endswith("_index"):
        nodes = np.broadcast_to(np.arange(s, dtype=float), x.shape + (s,))
        pt = x - b
    elif scheme.endswith("_theta"):
        nodes = np.stack([np.asarray(omega)[b + k] for k in range(s)], axis=-1)
        pt = np.broadcast_to(np.asarray(om_pt, dtype=float), x.shape)
    else:
        raise ValueError("unknown interpolation scheme %r" % scheme)
    return b, fh_weights(nodes, pt, dd)


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
