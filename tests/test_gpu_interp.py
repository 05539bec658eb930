"""The theta-stencil schemes of Sec. 3.3 beyond the default Lagrange-in-index: Floater-Hormann
rational interpolation and both schemes on the theta values of the nodes, on the device
against the oracle (history integrals, two-time lookups, whole solves)."""
import numpy as np
import pytest

from gpu_common import frozen_case, need_gpu
from oracle import integrals as OI
from oracle import solver as OS
from oracle.model import Model
from paper_2604_06309_gb300.inputs import MIXED_34

pytestmark = pytest.mark.gpu

SCHEMES = [("fh_index", 3), ("fh_index", 0), ("lagrange_theta", 3), ("fh_theta", 2)]


@pytest.mark.parametrize("interp,d", SCHEMES)
@pytest.mark.parametrize("t_stage", ["last", "beyond"])
def test_history_integrals_match_oracle(interp, d, t_stage):
    need_gpu()
    from paper_2604_06309_gb300 import Solver
    L, s = 65, 6
    sv = Solver(MIXED_34, 0.5, L, 1e3, s=s, history_cap=60, interp=interp, fh_d=d)
    hist = frozen_case(sv, 31, 60, 300.0)
    t = hist[0][-1] * (1.0 if t_stage == "last" else 1.01)
    C, R = hist[1][-1], hist[3][-1]
    S, _ = sv.history_integrals(t, C, R)
    G = OI.Grid(L, 1e3, s, interp=interp, fh_d=d)
    Sref = OI.history_integrals(Model(MIXED_34, 0.5), G, OI.History(*hist), t, C, R)
    assert np.max(np.abs(S - Sref)) < 1e-11
    sv.close()


@pytest.mark.parametrize("interp,d", SCHEMES[:1] + SCHEMES[3:])
def test_solve_and_lookups_match_oracle_step_by_step(interp, d):
    need_gpu()
    from paper_2604_06309_gb300 import Solver
    kw = dict(s=6, history_cap=24, dt0=0.2, interp=interp, fh_d=d)
    g = Solver(MIXED_34, 0.5, 33, 100.0, **kw)
    o = OS.Solver(MIXED_34, 0.5, L=33, grid_t_max=100.0, **kw)
    assert g.integrate(2.0, 1e-8) == 0
    assert o.integrate(2.0, 1e-8) == 0
    tg, Cg, _, Rg, _ = g.get_history()
    assert np.array_equal(tg, o.hist.t)
    assert np.max(np.abs(Cg - o.hist.C)) < 1e-9 and np.max(np.abs(Rg - o.hist.R)) < 1e-9
    t, tp = np.array([2.0, 2.0, 1.7, 0.9]), np.array([0.0, 1.3, 1.69, 0.2])
    assert np.max(np.abs(g.get_C(t, tp) - o.get_C(t, tp))) < 1e-10
    assert np.max(np.abs(g.get_R(t, tp) - o.get_R(t, tp))) < 1e-10
    g.close()


def test_schemes_other_than_lagrange_index_need_fp64():
    need_gpu()
    from paper_2604_06309_gb300 import DMFEError, Solver
    for prec in ("df", "fp32"):
        with pytest.raises(DMFEError) as e:
            Solver(MIXED_34, 0.5, 33, 100.0, precision=prec, interp="fh_index")
        assert e.value.code == -8
    with pytest.raises(DMFEError) as e:
        Solver(MIXED_34, 0.5, 33, 100.0, s=4, interp="fh_index", fh_d=4)   # d > s - 1
    assert e.value.code == -1
