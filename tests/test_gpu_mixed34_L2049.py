"""The benchmark solve itself -- the mixed (3+4)-spin quench, T = 0.5, on the L = 2049 grid
for t_max = 1e5 with a 2049-slice store, s = 4, tol 1e-8 -- on the device from t = 0,
compared at t = 0.1 and t = 1 with the oracle's solve stored in
tests/golden/mixed34_T0.5_L2049.json (written by tests/golden/make_mixed34_quench.py 2049, which
calls only the oracle): identical step decisions, and C, R, E, mu within 1e-9."""
import json
import os

import numpy as np
import pytest

from gpu_common import need_gpu

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "mixed34_T0.5_L2049.json")


@pytest.mark.parametrize("precision", ["fp64", "df"])
def test_benchmark_solve_matches_oracle_at_checkpoints(precision):
    need_gpu()
    from paper_2604_06309_gb300 import Solver
    with open(GOLDEN) as f:
        g = json.load(f)
    c = g["case"]
    cols = np.array(g["columns"])
    sv = Solver({int(p): q for p, q in c["coefs"].items()}, c["T"], c["L"], c["grid_t_max"], s=c["s"],
                history_cap=c["history_cap"], precision=precision)
    for cp in g["checkpoints"]:
        assert sv.integrate(cp["t"], c["tol"]) == 0
        tg, Cg, _, Rg, _ = sv.get_history()
        assert np.array_equal(tg, np.array(cp["slice_times"])), cp["t"]
        st = sv.stats()
        for k in ("steps_accepted", "steps_rejected", "sparsify_passes", "slices_removed"):
            assert st[k] == cp["stats"][k], (cp["t"], k)
        assert np.max(np.abs(Cg[-1][cols] - np.array(cp["C_cols"]))) < 1e-9
        assert np.max(np.abs(Rg[-1][cols] - np.array(cp["R_cols"]))) < 1e-9
        t, tp = np.array(cp["pairs"]).T
        assert np.max(np.abs(sv.get_C(t, tp) - np.array(cp["C_pairs"]))) < 1e-9
        assert np.max(np.abs(sv.get_R(t, tp) - np.array(cp["R_pairs"]))) < 1e-9
        _, _, _, mu, E = sv.get_row()
        assert abs(E - cp["E"]) < 1e-9 and abs(mu - cp["mu"]) < 1e-9
    sv.close()
