"""SSPRK(10,4) and the Dormand-Prince -> SSPRK(10,4) switch (Sec. 3.5) on the device,
step by step against the oracle, and in batches mixing both methods."""
import numpy as np
import pytest

from gpu_common import need_gpu
from oracle import solver as OS
from oracle.model import Model
from paper_2604_06309_gb300.inputs import MIXED_34, PURE_3

pytestmark = pytest.mark.gpu


def _pair(coefs, T, L, t_max_grid, cap, precision="fp64", **kw):
    from paper_2604_06309_gb300 import Solver
    g = Solver(coefs, T, L, t_max_grid, history_cap=cap, precision=precision, **kw)
    o = OS.Solver(coefs, T, L=L, grid_t_max=t_max_grid, history_cap=cap, **kw)
    return g, o


def _compare_runs(g, o, tol_rows):
    tg, Cg, dCg, Rg, dRg = g.get_history()
    assert len(tg) == o.hist.N
    assert np.array_equal(tg, o.hist.t)          # identical step decisions => identical times
    for a, b in ((Cg, o.hist.C), (dCg, o.hist.dC), (Rg, o.hist.R), (dRg, o.hist.dR)):
        assert np.max(np.abs(a - b)) < tol_rows
    st = g.stats()
    for k in ("steps_accepted", "steps_rejected", "sparsify_passes", "slices_removed"):
        assert st[k] == o.stats[k], k
    return st


@pytest.mark.parametrize("precision", ["fp64", "df"])
def test_ssprk104_matches_oracle_step_by_step(precision):
    need_gpu()
    g, o = _pair(PURE_3, 0.8, 33, 100.0, cap=400, precision=precision, integrator="ssprk104", dt0=0.01)
    assert g.integrate(1.5, 1e-8) == 0
    assert o.integrate(1.5, 1e-8) == 0
    st = _compare_runs(g, o, 1e-9)
    assert st["method"] == 2 and st["t_switch"] == -1.0
    assert st["step_graph"] == 2        # the SSPRK stages ran in the conditional node
    # ten stage evaluations per trial step
    assert st["stages"] == 10 * (st["steps_accepted"] + st["steps_rejected"])
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "df"])
def test_switch_matches_oracle_with_rejections_and_sparsification(precision):
    need_gpu()
    # dt0 = 0.3 forces rejections, cap = 40 sparsification passes, switch_dt = 0.035 a
    # switch early in the run
    g, o = _pair(MIXED_34, 0.5, 33, 100.0, cap=40, precision=precision, dt0=0.3, switch_dt=0.035)
    assert g.integrate(4.0, 1e-8) == 0
    assert o.integrate(4.0, 1e-8) == 0
    assert o.t_switch is not None and o.stats["steps_rejected"] >= 1 and o.stats["sparsify_passes"] >= 1
    st = _compare_runs(g, o, 1e-9)
    assert st["method"] == 2 and st["t_switch"] == o.t_switch
    assert st["rk_switch_dt"] == 0.035
    g.close()


def test_automatic_switch_step_matches_stability_estimate():
    need_gpu()
    from paper_2604_06309_gb300 import Solver
    for coefs in (MIXED_34, PURE_3, {2: 0.5}, {3: 0.4, 4: 0.1}):
        g = Solver(coefs, 0.5, 33, 100.0, history_cap=64)
        ref = OS.switch_dt_auto(Model(coefs, 0.5))
        assert abs(g.stats()["rk_switch_dt"] - ref) < 1e-12 * ref
        g.close()
    g = Solver({1: 0.5}, 0.5, 33, 100.0, history_cap=64)       # f'' = 0: never
    assert g.stats()["rk_switch_dt"] == np.inf
    g.close()
    g = Solver(MIXED_34, 0.5, 33, 100.0, history_cap=64, integrator="dp5")
    assert g.stats()["rk_switch_dt"] == np.inf and g.stats()["method"] == 1
    g.close()


def test_switch_through_async_steps_and_checkpoint(tmp_path):
    """dmfe_step launches graphs without reading the state: the device switches method
    inside the run; a checkpoint taken after the switch restores the SSPRK state."""
    need_gpu()
    from paper_2604_06309_gb300 import Solver
    g = Solver(PURE_3, 0.8, 33, 100.0, history_cap=200, switch_dt=0.015, dt0=0.01)
    g.step(400, 2.0, 1e-8)
    g.sync()
    o = OS.Solver(PURE_3, 0.8, L=33, grid_t_max=100.0, history_cap=200, switch_dt=0.015, dt0=0.01)
    assert o.integrate(2.0, 1e-8) == 0
    st = _compare_runs(g, o, 1e-9)
    assert st["method"] == 2 and st["t_switch"] == o.t_switch
    path = str(tmp_path / "ssp.ckp")
    g.checkpoint(path)
    r = Solver.restore(path)
    assert r.stats()["method"] == 2 and r.stats()["t_switch"] == o.t_switch
    assert g.integrate(3.0, 1e-8) == 0 and r.integrate(3.0, 1e-8) == 0
    for x, y in zip(g.get_history(), r.get_history()):
        assert np.array_equal(x, y)
    g.close()
    r.close()


@pytest.mark.parametrize("precision", ["fp64", "df"])
def test_batch_mixing_methods_is_bitwise_equal_to_solo_runs(precision):
    need_gpu()
    from paper_2604_06309_gb300 import Batch, Solver
    tol = 1e-8
    cases = [  # (f, T, L, cap, t_max, integrator kwargs)
        (MIXED_34, 0.5, 33, 24, 2.0, dict(integrator="ssprk104")),
        (PURE_3, 0.8, 65, 64, 1.5, dict(integrator="dp5")),
        ({3: 0.4, 4: 0.1}, 0.3, 129, 48, 2.5, dict(switch_dt=0.02, dt0=0.01)),
    ]
    b = Batch(4, 129, 64, precision=precision)
    slots = [b.add(f, T, L, 1e3, tmax, tol, history_cap=cap, **kw) for (f, T, L, cap, tmax, kw) in cases]
    b.run()
    status, t, running = b.poll()
    assert running == 0
    for (f, T, L, cap, tmax, kw), k in zip(cases, slots):
        assert status[k] == 1 and t[k] == tmax
        sv = Solver(f, T, L, 1e3, history_cap=cap, precision=precision, hi_chunk=L, **kw)
        assert sv.integrate(tmax, tol) == 0
        for x, y in zip(b.solver(k).get_history(), sv.get_history()):
            assert np.array_equal(x, y)
        a, s = b.solver(k).stats(), sv.stats()
        assert a["method"] == s["method"] and a["t_switch"] == s["t_switch"]
        sv.close()
    assert b.solver(slots[2]).stats()["t_switch"] > 0
    b.close()
