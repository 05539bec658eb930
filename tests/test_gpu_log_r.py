"""The optional logarithmic interpolation of the response history (App. A) on the FP64
device path against the oracle: history integrals on frozen histories (with and without
regions where R is not positive, which keep the linear interpolation), a whole solve with
two-time lookups, and checkpoint/restore of the log-R coefficient tables."""
import numpy as np
import pytest

from gpu_common import need_gpu
from oracle import integrals as OI
from oracle import solver as OS
from oracle.model import Model
from paper_2604_06309_gb300.inputs import MIXED_34, geometric_times, synthetic_history

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shift", [0.0, 0.05])
@pytest.mark.parametrize("t_stage", ["last", "beyond"])
def test_history_integrals_match_oracle(shift, t_stage):
    need_gpu()
    from paper_2604_06309_gb300 import Solver
    L, s = 65, 6
    sv = Solver(MIXED_34, 0.5, L, 1e3, s=s, history_cap=60, log_r=True)
    times = geometric_times(60, 1e-2, 300.0)
    C, dC, R, dR = synthetic_history(31, times, sv.theta, sv.omega)
    R = R - shift        # shift > 0: about a quarter of the stored R values are negative
    sv.set_history(times, C, dC, R, dR)
    t = times[-1] * (1.0 if t_stage == "last" else 1.01)
    S, _ = sv.history_integrals(t, C[-1], R[-1])
    H = OI.History(times, C, dC, R, dR)
    m = Model(MIXED_34, 0.5)
    Sref = OI.history_integrals(m, OI.Grid(L, 1e3, s, log_r=True), H, t, C[-1], R[-1])
    Slin = OI.history_integrals(m, OI.Grid(L, 1e3, s), H, t, C[-1], R[-1])
    assert np.max(np.abs(Sref - Slin)) > 1e-6       # the log-R reading changes the sums
    assert np.max(np.abs(S - Sref)) < 1e-11
    sv.close()


def test_solve_and_lookups_match_oracle_step_by_step():
    need_gpu()
    from paper_2604_06309_gb300 import Solver
    # small store and a large first step: sparsification passes and rejections
    kw = dict(s=4, history_cap=24, dt0=0.3, log_r=True)
    g = Solver(MIXED_34, 0.5, 33, 100.0, **kw)
    o = OS.Solver(MIXED_34, 0.5, L=33, grid_t_max=100.0, **kw)
    assert g.integrate(2.0, 1e-8) == 0
    assert o.integrate(2.0, 1e-8) == 0
    assert o.stats["sparsify_passes"] >= 1
    tg, Cg, _, Rg, _ = g.get_history()
    assert np.array_equal(tg, o.hist.t)
    assert np.max(np.abs(Cg - o.hist.C)) < 1e-9 and np.max(np.abs(Rg - o.hist.R)) < 1e-9
    t, tp = np.array([2.0, 2.0, 1.7, 0.9, 1.3]), np.array([0.0, 1.3, 1.69, 0.2, 1.3])
    assert np.max(np.abs(g.get_C(t, tp) - o.get_C(t, tp))) < 1e-10
    assert np.max(np.abs(g.get_R(t, tp) - o.get_R(t, tp))) < 1e-10
    _, _, _, _, E = g.get_row()
    assert abs(E - o.E) < 1e-10
    g.close()


def test_checkpoint_restore_rebuilds_log_tables(tmp_path):
    need_gpu()
    from paper_2604_06309_gb300 import Solver
    a = Solver(MIXED_34, 0.5, 33, 100.0, history_cap=24, log_r=True)
    b = Solver(MIXED_34, 0.5, 33, 100.0, history_cap=24, log_r=True)
    assert a.integrate(1.0, 1e-8) == 0 and b.integrate(1.0, 1e-8) == 0
    path = str(tmp_path / "ck.bin")
    a.checkpoint(path)
    a.close()
    r = Solver.restore(path)
    assert r.integrate(2.0, 1e-8) == 0 and b.integrate(2.0, 1e-8) == 0
    for x, y in zip(r.get_history(), b.get_history()):
        assert np.array_equal(x, y)
    r.close()
    b.close()


def test_log_r_needs_fp64():
    need_gpu()
    from paper_2604_06309_gb300 import DMFEError, Solver
    for prec in ("df", "fp32"):
        with pytest.raises(DMFEError) as e:
            Solver(MIXED_34, 0.5, 33, 100.0, precision=prec, log_r=True)
        assert e.value.code == -8


def test_batches_and_servers_refuse_log_r():
    need_gpu()
    from paper_2604_06309_gb300 import Batch, DMFEError, Server
    b = Batch(2, 65, 32)
    with pytest.raises(DMFEError) as e:
        b.add(MIXED_34, 0.5, 65, 100.0, 1.0, 1e-8, history_cap=32, log_r=True)
    assert e.value.code == -8
    b.add(MIXED_34, 0.5, 65, 100.0, 1.0, 1e-8, history_cap=32)     # the slot is still free
    b.close()
    srv = Server(2, 65, 32, hbm_budget=1 << 30)
    with pytest.raises(DMFEError) as e:
        srv.submit(MIXED_34, 0.5, 65, 100.0, 1.0, 1e-8, history_cap=32, log_r=True)
    assert e.value.code == -8
    srv.stop()
