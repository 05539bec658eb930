"""History integrals, mu(t), E(t) and the right-hand side (Secs. 2.1, 3.3, 3.4).

Fields on the two-time grid (Sec. 3.1): Cf(t, theta) = C(t, theta t) and
Rf(t, theta) = R(t, theta t). The history stores, for each slice t_n, the rows
Cf, dCf/dt|theta, Rf, dRf/dt|theta on the theta grid (Sec. 3.2, last paragraph).

Equations (Eq. genericDMFE with the kernels of Sec. 2.1; reading: the -mu(t) C and
-mu(t) R terms that Eq. genericDMFE leaves out are restored, since mu is defined
there and C(t,t) = 1 needs them):

    d1 C(t,t') = -mu(t) C + int_0^t K(t,s) C(s,t') ds + int_0^t' D(t,s) R(t',s) ds + F_C(t,t')
    d1 R(t,t') = -mu(t) R + int_t'^t K(t,s) R(s,t') ds
    mu(t)      = T + int_0^t [K C + D R](t,s) ds + F_C(t,t)
    E(t)       = -int_0^t f'(C(t,s)) R(t,s) ds - beta0 f(C(t,0))

The solver advances Cf, Rf at fixed theta, so it needs the total derivative
d/dt C(t, theta t) = d1 C + theta d2 C (likewise R). Reading: d2 (the derivative in
the second time) is taken from the DMFE themselves, not from a numerical theta
derivative (which would make the explicit Runge-Kutta scheme stiff, with
eigenvalues ~ 1/(t dtheta_min)):

    d2 C(t,t') = [d1 C](t', t)      (C symmetric; first argument t' < t, so the
                 = -mu(t') C(t,t') + int_0^t' K(t',s) C(s,t) ds
                   + int_0^t D(t',s) R(t,s) ds + 2 T R(t,t') + beta0 f'(C(t',0)) C(t,0)
    d2 R(t,t') = mu(t') R(t,t') - int_t'^t R(t,s) K(s,t') ds      (adjoint equation)
    mu(t')     = T + int_0^t' [K C + D R](t',s) ds + F_C(t',t')

All integrals map to the fixed theta grid (Sec. 3.3): with t' = theta_j t,
phi1_ij = theta_i theta_j on [0, t'] (ds = t theta_j dtheta_i) and
phi2_ij = theta_j + (1 - theta_j) theta_i on [t', t] (ds = t (1 - theta_j) dtheta_i).
The values come from three interpolations (Sec. 3.3):

    A   current row at phi1 or phi2 (index Lagrange stencil):    K, D, Cf, Rf
    B1  Cf(theta_j t, theta_i), Rf(theta_j t, theta_i): on-grid theta, Hermite in t
    B2  Cf(phi2 t, theta_j / phi2), Rf(...): Lagrange in theta on the two slices
        around phi2 t, then Hermite in t

and the quadrature is I = sum_i nu_i A_ij B_ij (Eq. int; reading: j is the output
index and i the summation index, and the Jacobians theta_j, 1 - theta_j are kept).

Times inside the current step (t_last < tau <= t, reading): the quadratic through
(y_last, y'_last) at t_last and the current row at t. Times below t_last use the
cubic Hermite on the stored interval containing them.

Outputs of ``history_integrals`` (rows of S, each of length L, before the factors
t theta_j or t (1 - theta_j)):

    S[0] = sum nu K_A1 Cf_B1          int_0^t'  K(t,s) C(t',s)
    S[1] = sum nu K_A2 Cf_B2          int_t'^t  K(t,s) C(s,t')
    S[2] = sum nu D_A1 Rf_B1          int_0^t'  D(t,s) R(t',s)
    S[3] = sum nu K_A2 Rf_B2          int_t'^t  K(t,s) R(s,t')
    S[4] = sum nu f''(Cf_B1) Rf_B1 Cf_A1     int_0^t' K(t',s) C(t,s)
    S[5] = sum nu f'(Cf_B1) Rf_A1            int_0^t' D(t',s) R(t,s)
    S[6] = sum nu f'(Cf_B2) Rf_A2            int_t'^t D(t',s) R(t,s)
    S[7] = sum nu f''(Cf_B2) Rf_B2 Rf_A2     int_t'^t R(t,s) K(s,t')
    S[8] = sum nu [f''(Cf_B1) Cf_B1 + f'(Cf_B1)] Rf_B1   mu(t') - T
    S[9] = Cf_B1 at theta_i = 0, i.e. C(t', 0)          (for F_C)

Pins: tests/test_oracle_integrals.py (exact p = 2 solution: the right-hand side
built from exact histories matches the analytic derivative; f = 0 closed form;
mu = T - p E for pure models; the theta = 1 value d1 C(t, t^-) = -T).
"""

import numpy as np

from .interp import lagrange_stencil, scheme_stencil, hermite

NS = 10  # number of rows of S


class Grid:
    """The theta grid, its complement, the weights nu and the three stencil sets.

    The stencil positions (Sec. 3.3) of output rows j are produced by ``stencils(js)``;
    they depend only on the grid and are kept for small L (the "precomputed" weights
    of the paper), recomputed per block of rows otherwise.
    """

    CACHE_MAX_L = 1024

    def __init__(self, L, t_max, s=4, alpha=0.0, delta=0.0, interp="lagrange_index", fh_d=3, log_r=False):
        from . import grid as g
        from .quadrature import spline_weights
        from .interp import SCHEMES
        if interp not in SCHEMES:
            raise ValueError("unknown interpolation scheme %r" % interp)
        self.interp, self.fh_d = interp, int(fh_d)
        self.log_r = bool(log_r)  # logarithmic interpolation of the response history
        self.L, self.s = int(L), int(s)
        self.t_max, self.alpha, self.delta = float(t_max), float(alpha), float(delta)
        self.gamma = g.gamma_from_tmax(t_max)
        self.theta, self.omega = g.theta_grid(self.L, self.gamma, alpha, delta)
        self.nu = spline_weights(self.theta)
        self._cache = self.positions(slice(0, self.L)) if self.L <= self.CACHE_MAX_L else None

    def positions(self, js):
        """(phi2, x1, x2, x3, o1, o2, o3) for output rows js: fractional indices of phi1,
        phi2, psi and their complements 1 - phi1, 1 - phi2, 1 - psi."""
        from . import grid as g
        th, om = self.theta, self.omega
        thj, omj = th[js][:, None], om[js][:, None]  # output index j along axis 0
        thi, omi = th[None, :], om[None, :]          # summation index i along axis 1
        # phi1 = theta_i theta_j, 1 - phi1 = omega_i + theta_i omega_j
        phi1, ophi1 = thj * thi, omi + thi * omj
        # phi2 = theta_j + omega_j theta_i, 1 - phi2 = omega_j omega_i
        phi2, ophi2 = thj + omj * thi, omj * omi
        # psi = theta_j / phi2 (0 where phi2 = 0), 1 - psi = omega_j theta_i / phi2
        safe = np.where(phi2 > 0, phi2, 1.0)
        psi = np.where(phi2 > 0, thj / safe, 0.0)
        opsi = np.where(phi2 > 0, omj * thi / safe, 1.0)
        fi = lambda a, b: g.frac_index(a, b, self.L, self.gamma, self.alpha, self.delta)
        return phi2, fi(phi1, ophi1), fi(phi2, ophi2), fi(psi, opsi), ophi1, ophi2, opsi

    def stencil_at(self, x, om):
        """(base, weights) of the grid's interpolation scheme at fractional index x whose
        point has complement om = 1 - theta."""
        return scheme_stencil(x, om, self.omega, self.L, self.s, self.interp, self.fh_d)

    def stencils(self, js):
        """(phi2, st1, st2, st3) for rows js; st = (base, weights) of the grid's scheme."""
        if self._cache is not None:
            phi2, x1, x2, x3, o1, o2, o3 = (a[js] for a in self._cache)
        else:
            phi2, x1, x2, x3, o1, o2, o3 = self.positions(js)
        return phi2, self.stencil_at(x1, o1), self.stencil_at(x2, o2), self.stencil_at(x3, o3)


class History:
    """Stored slices t_n (t_0 = 0, increasing) with rows C, dC, R, dR of shape [N, L]."""

    def __init__(self, t, C, dC, R, dR):
        self.t = np.array(t, dtype=float)
        self.C, self.dC = np.array(C, dtype=float), np.array(dC, dtype=float)
        self.R, self.dR = np.array(R, dtype=float), np.array(dR, dtype=float)

    @property
    def N(self):
        return len(self.t)

    def copy(self):
        return History(self.t, self.C, self.dC, self.R, self.dR)

    def keep(self, mask):
        return History(self.t[mask], self.C[mask], self.dC[mask], self.R[mask], self.dR[mask])

    def append(self, t, C, dC, R, dR):
        return History(np.append(self.t, t), np.vstack([self.C, C]), np.vstack([self.dC, dC]),
                       np.vstack([self.R, R]), np.vstack([self.dR, dR]))


def _gather(rows, n, b, w):
    """sum_k w_k rows[n, b + k] (w None: the on-grid value rows[n, b])."""
    if w is None:
        return rows[n, b]
    return sum(w[..., k] * rows[n, b + k] for k in range(w.shape[-1]))


def _gather_row(row, b, w):
    if w is None:
        return row[b]
    return sum(w[..., k] * row[b + k] for k in range(w.shape[-1]))


def _positive(rows, n, b, w):
    """True where every stencil value rows[n, b + k] (or rows[n, b]) is positive."""
    if w is None:
        return rows[n, b] > 0
    return np.all(np.stack([rows[n, b + k] > 0 for k in range(w.shape[-1])]), axis=0)


def _positive_row(row, b, w):
    if w is None:
        return row[b] > 0
    return np.all(np.stack([row[b + k] > 0 for k in range(w.shape[-1])]), axis=0)


def _safe_log(x):
    return np.log(np.where(x > 0, x, 1.0))


def lookup(hist, tau, b, w, t_cur, C_cur, R_cur, log_r=False):
    """(Cf, Rf) at times tau and theta positions (b, w) from the history (Sec. 3.3).

    b, w: stencil in the theta index (w None: on-grid column b). tau, b and w must
    broadcast together. tau <= t_cur is required.

    log_r (the optional logarithmic interpolation of the response history, App. A):
    where every stencil value of R on the slices involved is positive, R is
    interpolated as exp of the same interpolant applied to log R with the scaled
    derivative R'/R; elsewhere the linear interpolation is kept.
    """
    tau = np.asarray(tau, dtype=float)
    tau, b = np.broadcast_arrays(tau, b)
    N = hist.N
    tl = hist.t[-1]
    ext = (t_cur > tl) & (tau > tl)
    outC = np.empty(tau.shape)
    outR = np.empty(tau.shape)
    if log_r:
        lR, ldR = _safe_log(hist.R), hist.dR / np.where(hist.R > 0, hist.R, 1.0)
        lRc = _safe_log(np.asarray(R_cur, dtype=float))
    if np.any(ext):
        bb = b[ext]
        ww = None if w is None else np.broadcast_to(w, b.shape + w.shape[-1:])[ext]
        h = t_cur - tl
        sg = tau[ext] - tl
        quad = lambda y0, d0, y1: y0 + d0 * sg + (y1 - y0 - d0 * h) / (h * h) * sg * sg
        for rows, drows, cur, out in ((hist.C, hist.dC, C_cur, outC), (hist.R, hist.dR, R_cur, outR)):
            out[ext] = quad(_gather(rows, N - 1, bb, ww), _gather(drows, N - 1, bb, ww), _gather_row(cur, bb, ww))
        if log_r:
            pos = _positive(hist.R, N - 1, bb, ww) & _positive_row(np.asarray(R_cur), bb, ww)
            lv = np.exp(quad(_gather(lR, N - 1, bb, ww), _gather(ldR, N - 1, bb, ww), _gather_row(lRc, bb, ww)))
            outR[ext] = np.where(pos, lv, outR[ext])
    inn = ~ext
    if np.any(inn):
        bb = b[inn]
        ww = None if w is None else np.broadcast_to(w, b.shape + w.shape[-1:])[inn]
        ti = tau[inn]
        if N == 1:
            outC[inn] = _gather(hist.C, 0, bb, ww)
            outR[inn] = _gather(hist.R, 0, bb, ww)
            if log_r:
                outR[inn] = np.where(_positive(hist.R, 0, bb, ww), np.exp(_gather(lR, 0, bb, ww)), outR[inn])
        else:
            n = np.clip(np.searchsorted(hist.t, ti, side="right") - 1, 0, N - 2)
            h = hist.t[n + 1] - hist.t[n]
            sig = (ti - hist.t[n]) / h
            herm = lambda rows, drows: hermite(_gather(rows, n, bb, ww), _gather(drows, n, bb, ww),
                                              _gather(rows, n + 1, bb, ww), _gather(drows, n + 1, bb, ww), h, sig)
            outC[inn] = herm(hist.C, hist.dC)
            outR[inn] = herm(hist.R, hist.dR)
            if log_r:
                pos = _positive(hist.R, n, bb, ww) & _positive(hist.R, n + 1, bb, ww)
                outR[inn] = np.where(pos, np.exp(herm(lR, ldR)), outR[inn])
    return outC, outR


def row_prep(model, grid, t, C, R):
    """K, D on the current row, mu(t) and E(t) (Sec. 2.1; integrals by nu)."""
    K = model.fpp(C) * R
    D = model.fp(C)
    mu = model.T + t * np.sum(grid.nu * (K * C + D * R)) + model.beta0 * model.fp(C[0]) * C[0]
    E = -t * np.sum(grid.nu * model.fp(C) * R) - model.beta0 * model.f(C[0])
    return K, D, mu, E


def history_integrals(model, grid, hist, t, C, R, js=None, j_chunk=256):
    """The NS x L sums S of the module docstring for the stage at time t with row (C, R).

    js: optional list of output rows; the other columns of S are left at zero.
    """
    L = grid.L
    nu = grid.nu
    K, D, _, _ = row_prep(model, grid, t, C, R)
    S = np.zeros((NS, L))
    cols = np.arange(L)
    rows = np.arange(L) if js is None else np.asarray(js)
    for c0 in range(0, len(rows), j_chunk):
        jr = rows[c0:c0 + j_chunk]
        thj = grid.theta[jr][:, None]
        phi2, (b1, w1), (b2, w2), (b3, w3) = grid.stencils(jr)
        # A: current row at phi1 and phi2
        K_A1, D_A1 = _gather_row(K, b1, w1), _gather_row(D, b1, w1)
        C_A1, R_A1 = _gather_row(C, b1, w1), _gather_row(R, b1, w1)
        K_A2, R_A2 = _gather_row(K, b2, w2), _gather_row(R, b2, w2)
        # B1: on-grid theta_i at time theta_j t
        C_B1, R_B1 = lookup(hist, thj * t, cols[None, :], None, t, C, R, grid.log_r)
        # B2: theta position psi_ij at time phi2_ij t
        C_B2, R_B2 = lookup(hist, phi2 * t, b3, w3, t, C, R, grid.log_r)
        fpp1, fp1 = model.fpp(C_B1), model.fp(C_B1)
        fpp2, fp2 = model.fpp(C_B2), model.fp(C_B2)
        terms = (K_A1 * C_B1, K_A2 * C_B2, D_A1 * R_B1, K_A2 * R_B2,
                 fpp1 * R_B1 * C_A1, fp1 * R_A1, fp2 * R_A2, fpp2 * R_B2 * R_A2,
                 (fpp1 * C_B1 + fp1) * R_B1)
        for r, term in enumerate(terms):
            S[r, jr] = np.sum(nu[None, :] * term, axis=1)
        S[9, jr] = C_B1[:, 0]
    return S


def assemble_rhs(model, grid, t, C, R, S, mu):
    """Total derivatives (dCf/dt, dRf/dt) at fixed theta from the sums S (module docstring).

    The diagonal theta = 1 is pinned: C(t,t) = 1 and R(t,t^-) = 1, so its derivative is 0.
    """
    T, b0 = model.T, model.beta0
    th, om = grid.theta, grid.omega
    C0 = C[0]
    d1C = -mu * C + t * (th * (S[0] + S[2]) + om * S[1]) + b0 * model.fp(C0) * S[9]
    d1R = -mu * R + t * om * S[3]
    mu_p = T + t * th * S[8] + b0 * model.fp(S[9]) * S[9]
    d2C = -mu_p * C + t * (th * (S[4] + S[5]) + om * S[6]) + 2.0 * T * R + b0 * model.fp(S[9]) * C0
    d2R = mu_p * R - t * om * S[7]
    dC = d1C + th * d2C
    dR = d1R + th * d2R
    dC[-1] = 0.0
    dR[-1] = 0.0
    return dC, dR


def rhs(model, grid, hist, t, C, R):
    """Right-hand side of the theta-grid ODE for the stage (t, C, R); returns (dC, dR, mu, E)."""
    _, _, mu, E = row_prep(model, grid, t, C, R)
    if t == 0.0:
        # all integrals carry a factor t; C(t',0) = C(0,0) = 1
        S = np.zeros((NS, grid.L))
        S[9] = 1.0
    else:
        S = history_integrals(model, grid, hist, t, C, R)
    dC, dR = assemble_rhs(model, grid, t, C, R, S, mu)
    return dC, dR, mu, E
