"""Pins for oracle/solver.py (Secs. 3.1, 3.5, 3.6) against closed forms and brute force."""
import numpy as np
import pytest

from oracle import closed_forms as cf
from oracle import solver as S
from oracle.integrals import Grid, History
from oracle.model import Model


def test_dormand_prince_tableau_is_consistent():
    for st in range(1, 7):
        assert abs(sum(S.DP_A[st]) - S.DP_C[st]) < 1e-15
    assert abs(S.DP_B5.sum() - 1) < 1e-15 and abs(S.DP_B4.sum() - 1) < 1e-15
    # order conditions up to 4 for both weight vectors: sum b c^k = 1/(k+1)
    for b in (S.DP_B5, S.DP_B4):
        for k in range(4):
            assert abs(b @ S.DP_C ** k - 1 / (k + 1)) < 1e-14


def test_dp5_local_orders_on_scalar_ode():
    f = lambda t, y: np.array([-y[0] + np.sin(3 * t)])
    exact = lambda t: (np.exp(-t) * (1 + 3 / 10) + (np.sin(3 * t) - 3 * np.cos(3 * t)) / 10)
    errs, ests = [], []
    hs = [0.2, 0.1, 0.05, 0.025]
    for h in hs:
        y0 = np.array([exact(0.3)])
        y1, est, _ = S.dp5_step(f, 0.3, y0, h, f(0.3, y0))
        errs.append(abs(y1[0] - exact(0.3 + h)))
        ests.append(abs(est[0]))
    slope = lambda e: np.polyfit(np.log(hs), np.log(e), 1)[0]
    assert slope(errs) > 5.3          # local error of the 5th-order solution, O(h^6)
    assert 4.7 < slope(ests) < 5.6    # embedded estimate, O(h^5)


def test_free_model_solution():
    sv = S.Solver({2: 0.0}, 0.6, L=33, grid_t_max=10.0, history_cap=400)
    assert sv.integrate(2.0, 1e-9) == S.OK
    # the stored rows are exact to rounding ...
    assert np.max(np.abs(sv.hist.C[-1] - np.exp(-0.6 * 2.0 * sv.grid.omega))) < 1e-13
    # ... and off-grid reads carry only the theta-interpolation error of L = 33, s = 4
    t, tp = np.array([2.0, 2.0, 1.3]), np.array([0.0, 1.5, 0.2])
    assert np.max(np.abs(sv.get_C(t, tp) - np.exp(-0.6 * (t - tp)))) < 3e-5


@pytest.fixture(scope="module")
def p2_run():
    sv = S.Solver({2: 0.5}, 0.0, L=65, grid_t_max=100.0, s=6, history_cap=4000)
    st = sv.integrate(5.0, 1e-10)
    return st, sv


def test_p2_energy_matches_exact(p2_run):
    """Sec. 4.2: E_sim - E_exact for the pure 2-spin quench to T = 0."""
    st, sv = p2_run
    assert st == S.OK
    assert abs(sv.E - cf.p2_E(5.0)) < 1e-7


def test_p2_two_time_functions_match_exact(p2_run):
    _, sv = p2_run
    t = np.array([5.0, 5.0, 5.0, 3.3, 1.0])
    tp = np.array([4.9, 2.0, 0.0, 1.1, 0.5])
    # stored rows: solver error only; off-grid reads add the L = 65 interpolation error
    G = sv.grid
    assert np.max(np.abs(sv.hist.C[-1] - cf.p2_C(5.0, 5.0 * G.theta))) < 1e-6
    assert np.max(np.abs(sv.hist.R[-1] - cf.p2_R(5.0, 5.0 * G.theta))) < 1e-6
    assert np.max(np.abs(sv.get_C(t, tp) - cf.p2_C(t, tp))) < 3e-6
    assert np.max(np.abs(sv.get_R(t, tp) - cf.p2_R(t, tp))) < 3e-6


def test_structural_invariants(p2_run):
    _, sv = p2_run
    ts = np.array([0.5, 1.7, 5.0])
    assert np.max(np.abs(sv.get_C(ts, ts) - 1)) < 1e-14            # C(t,t) = 1
    assert np.max(np.abs(sv.get_R(ts, ts) - 1)) < 1e-14            # R(t,t^-) = 1
    assert np.all(sv.get_R(np.array([1.0, 2.0]), np.array([1.5, 4.0])) == 0)  # causality
    assert np.all(sv.hist.C <= 1 + 1e-12)
    # random initial condition: C(t,0) = R(t,0)
    assert np.max(np.abs(sv.hist.C[:, 0] - sv.hist.R[:, 0])) < 1e-10


def test_agrees_with_brute_force_uniform_grid_solver():
    """p = 3, T = 0.8: Richardson-extrapolated O(N^3) solver vs the non-uniform oracle."""
    m = Model({3: 0.5}, 0.8)
    hs = [0.04, 0.02, 0.01]
    bf = [cf.uniform_solve(m, 2.0, h) for h in hs]
    sv = S.Solver({3: 0.5}, 0.8, L=65, grid_t_max=100.0, s=6, history_cap=4000)
    assert sv.integrate(2.0, 1e-10) == S.OK
    for ta, tb in [(2.0, 1.0), (2.0, 0.0), (2.0, 1.6), (1.2, 0.4)]:
        for k, which in ((0, "C"), (1, "R")):
            v = [r[k][int(round(ta / h)), int(round(tb / h))] for r, h in zip(bf, hs)]
            r1, r2 = (4 * v[1] - v[0]) / 3, (4 * v[2] - v[1]) / 3
            got = sv.get_C(ta, tb)[0] if which == "C" else sv.get_R(ta, tb)[0]
            assert abs(got - r2) < 3 * abs(r2 - r1) + 1e-6, (ta, tb, which, got, r2)


@pytest.mark.slow
def test_equilibrium_fdt_above_Td():
    """p = 3, T = 0.8 > T_d: C(t, t - tau) -> C_eq(tau) and R -> -(1/T) dC_eq/dtau."""
    T = 0.8
    m = Model({3: 0.5}, T)
    tau = np.linspace(0.0, 4.0, 21)
    Ceq, dCeq, est = cf.equilibrium_C_richardson(m.fp, T, 4.0, 0.02)
    Ceq, dCeq = Ceq[::10], dCeq[::10]
    assert est < 1e-7
    sv = S.Solver({3: 0.5}, T, L=65, grid_t_max=100.0, s=6, history_cap=4000)
    errs, eerr = [], []
    for t in [8.0, 16.0]:
        assert sv.integrate(t, 1e-9) == S.OK
        ec = np.max(np.abs(sv.get_C(t, t - tau) - Ceq))
        er = np.max(np.abs(sv.get_R(t, t - tau) + dCeq / T))
        errs.append(max(ec, er))
        eerr.append(abs(sv.E - (-0.5 / T)))   # E_eq = -f(1)/T
    # the approach to equilibrium: both distances shrink several-fold from t = 8 to 16
    assert errs[1] < 0.4 * errs[0] and errs[1] < 2e-2
    assert eerr[1] < 0.5 * eerr[0] and eerr[1] < 1e-2


def _cubic_history(N=30, L=9):
    t = np.linspace(0.0, 3.0, N)
    rng = np.random.default_rng(5)
    c = rng.normal(size=(4, L))
    P = lambda tt: c[0] + c[1] * tt + c[2] * tt ** 2 + c[3] * tt ** 3
    dP = lambda tt: c[1] + 2 * c[2] * tt + 3 * c[3] * tt ** 2
    C = np.array([P(x) for x in t])
    dC = np.array([dP(x) for x in t])
    return History(t, C, dC, 0.5 * C, 0.5 * dC)


def test_sparsify_removes_slices_lying_on_cubics_with_skip_rule():
    H = _cubic_history()
    eps = S.sparsify_residuals(H)
    assert np.max(eps[1:-1]) < 1e-12
    stats = dict(sparsify_passes=0, slices_removed=0, forced_removals=0, max_eps_sparse=0.0)
    H2, ran = S.sparsify_pass(H, 1e-8, stats)
    assert ran
    # candidates 1..N-12 all pass: remove 1, skip 2, remove 3, ...
    removed = sorted(set(H.t) - set(H2.t))
    expect = H.t[1:H.N - 11:2]
    assert np.allclose(removed, expect)
    assert stats["forced_removals"] == 0


def test_sparsify_greedy_skip_and_forced_removal():
    H = _cubic_history()
    # break the cubic at slices 5 and 8 so that n = 4..6 and 7..9 fail
    H.C[5] += 1e-3
    H.C[8] += 1e-3
    eps = S.sparsify_residuals(H)
    ok = eps < 1e-9
    assert not ok[4] and not ok[5] and not ok[6] and ok[3] and ok[10]
    H2, _ = S.sparsify_pass(H, 1e-8)
    kept = np.isin(H.t, H2.t)
    scan, n = [], 1
    while n <= H.N - 12:
        if ok[n]:
            scan.append(n)
            n += 2
        else:
            n += 1
    assert sorted(np.where(~kept)[0]) == scan
    # nothing removable: the smallest residual is force-removed
    H3 = _cubic_history()
    H3.C[1:-1] += np.random.default_rng(0).normal(scale=1e-2, size=H3.C[1:-1].shape)
    st = dict(sparsify_passes=0, slices_removed=0, forced_removals=0, max_eps_sparse=0.0)
    H4, _ = S.sparsify_pass(H3, 1e-8, st)
    assert H4.N == H3.N - 1 and st["forced_removals"] == 1
    e3 = S.sparsify_residuals(H3)
    assert H3.t[1 + np.argmin(e3[1:H3.N - 11])] not in H4.t


def test_sparsify_selection_equals_the_run_parity_rule():
    """The greedy remove-n-skip-n+1 scan of Sec. 3.6 restated without a scan: within every
    maximal run of consecutive removable candidates (eps < tol/10, 1 <= n <= N-12) the
    removed slices are the run's first, third, fifth, ... members. Random breaks of a
    cubic history give random run patterns."""
    rng = np.random.default_rng(11)
    for _ in range(20):
        H = _cubic_history()
        broken = rng.choice(np.arange(1, H.N - 1), size=rng.integers(1, 8), replace=False)
        H.C[broken] += 1e-3
        eps = S.sparsify_residuals(H)
        last = H.N - 12
        ok = np.zeros(H.N, dtype=bool)
        ok[1:last + 1] = eps[1:last + 1] < 1e-9
        expect = []
        n = 1
        while n <= last:
            if not ok[n]:
                n += 1
                continue
            e = n
            while e + 1 <= last and ok[e + 1]:
                e += 1
            expect += list(range(n, e + 1, 2))
            n = e + 1
        H2, _ = S.sparsify_pass(H, 1e-8)
        got = sorted(np.where(~np.isin(H.t, H2.t))[0])
        if expect:
            assert got == expect
        else:   # nothing removable: one forced removal
            assert len(got) == 1


def test_two_passes_on_a_cubic_history_remove_alternate_survivors():
    """Every residual of a history lying on one cubic is zero, so each pass of the greedy
    scan removes the candidates 1, 3, 5, ... of the history it is given (candidates are
    slices 1 .. N-12): ceil((N - 12) / 2) slices. A second pass (reading R16: passes are
    repeated scans of the thinned history) does the same on the survivors."""
    H = _cubic_history(N=40)
    st = dict(sparsify_passes=0, slices_removed=0, forced_removals=0, max_eps_sparse=0.0)
    H1, ran1 = S.sparsify_pass(H, 1e-8, st, force=False)
    H2, ran2 = S.sparsify_pass(H1, 1e-8, st, force=False)
    assert ran1 and ran2
    r1 = -(-(H.N - 12) // 2)
    assert H1.N == H.N - r1
    r2 = -(-(H1.N - 12) // 2)
    assert H2.N == H1.N - r2
    assert np.array_equal(np.setdiff1d(H1.t, H2.t), H1.t[1:H1.N - 11:2])
    assert st == dict(sparsify_passes=2, slices_removed=r1 + r2, forced_removals=0, max_eps_sparse=st["max_eps_sparse"])


def test_a_pass_without_forcing_keeps_everything_when_nothing_qualifies():
    H = _cubic_history()
    H.C[1:-1] += np.random.default_rng(1).normal(scale=1e-2, size=H.C[1:-1].shape)
    st = dict(sparsify_passes=0, slices_removed=0, forced_removals=0, max_eps_sparse=0.0)
    H2, ran = S.sparsify_pass(H, 1e-8, st, force=False)
    assert ran and H2.N == H.N and np.array_equal(H2.t, H.t)
    assert st["sparsify_passes"] == 1 and st["slices_removed"] == 0 and st["forced_removals"] == 0
    # a history without candidates (N <= 12): no pass
    short = History(H.t[:12], H.C[:12], H.dC[:12], H.R[:12], H.dR[:12])
    assert S.sparsify_pass(short, 1e-8, st, force=False)[1] is False


def test_periodic_rounds_of_two_passes_stay_within_tolerance():
    """sparsify_every = 5, two passes per round, a store that never fills: rounds run after
    every fifth accepted step once there are candidates, and the solve stays close to the
    same solve without sparsification (each removal changes the stored integrals by less
    than tol / 10)."""
    kw = dict(L=33, grid_t_max=10.0, history_cap=1000)
    ref = S.Solver({3: 0.5}, 0.8, sparsify=False, **kw)
    assert ref.integrate(1.0, 1e-8) == S.OK
    sv = S.Solver({3: 0.5}, 0.8, sparsify_every=5, sparsify_passes=2, **kw)
    assert sv.integrate(1.0, 1e-8) == S.OK
    st = sv.stats
    assert st["forced_removals"] == 0 and st["slices_removed"] > 0
    assert sv.hist.N == st["steps_accepted"] + 1 - st["slices_removed"]
    # rounds after steps 5, 10, ...; a pass runs once there are 13 stored slices
    assert 0 < st["sparsify_passes"] <= 2 * (st["steps_accepted"] // 5)
    assert st["sparsify_passes"] % 2 == 0
    t = np.array([1.0, 1.0, 0.7, 0.5])
    tp = np.array([0.2, 0.9, 0.3, 0.49])
    assert np.max(np.abs(sv.get_C(t, tp) - ref.get_C(t, tp))) < 1e-7
    assert np.max(np.abs(sv.get_R(t, tp) - ref.get_R(t, tp))) < 1e-7
    assert abs(sv.E - ref.E) < 1e-7


def test_rejection_reverts_and_halves():
    sv = S.Solver({3: 0.5}, 0.8, L=33, grid_t_max=10.0, dt0=0.5, history_cap=100)
    assert sv.integrate(1.0, 1e-10) == S.OK
    assert sv.stats["steps_rejected"] >= 1
    first = sv.log[0]
    assert first[3] is False and first[1] == 0.5
    assert sv.log[1][1] == 0.25  # halved after the rejection
    assert sv.hist.N == sv.stats["steps_accepted"] + 1 - 0  # nothing to revert at the start


def test_step_underflow_status():
    sv = S.Solver({3: 0.5}, 0.8, L=33, grid_t_max=10.0, dt0=0.5, dt_min=0.3, history_cap=100)
    assert sv.integrate(1.0, 1e-12) == S.ERR_STEP_UNDERFLOW
