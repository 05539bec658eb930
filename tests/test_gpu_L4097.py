"""The largest configured grid, L = 4097 for grid t_max = 1e7 (the long-horizon
configuration), against the oracle.

1. Frozen histories of 4091 seeded slices (geometric times 1e-2 .. 9e6) in a 4097-slice
   store: the history integrals at the last slice time and at a stage time beyond it (the
   quadratic extension), in all three precisions, on sampled output rows including both
   edges. The FP64 kernel runs here with its largest shared-memory layout (stage row,
   slice times and reciprocal widths of 4098 slices, cell table: about 212 KB).
2. The quench itself from t = 0, step by step against the oracle's stored solve
   (tests/golden/mixed34_T0.5_L4097.json, written by
   tests/golden/make_mixed34_quench.py 4097, which calls only the oracle).
"""
import json
import os

import numpy as np
import pytest

from gpu_common import frozen_case, need_gpu
from oracle import integrals as OI
from oracle.model import Model
from paper_2604_06309_gb300.inputs import MIXED_34

pytestmark = pytest.mark.gpu

L = 4097
GRID_T_MAX = 1e7
ROWS = [0, 1, 2, 5, 100, 1000, 2048, 3000, 4000, 4090, L - 3, L - 2, L - 1]
# absolute bounds on S (whose entries reach ~5): FP64 differs from the oracle by summation
# order only; double-float carries a 48-bit significand; FP32 a 24-bit one with
# compensated sums (the kernel-level bounds of the smaller grids)
TOL = {"fp64": 1e-11, "df": 1e-10, "fp32": 3e-6}
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "mixed34_T0.5_L4097.json")


@pytest.mark.parametrize("precision", ["fp64", "df", "fp32"])
def test_frozen_history_4091_slices_sampled_rows(precision):
    need_gpu()
    from paper_2604_06309_gb300 import Solver
    sv = Solver(MIXED_34, 0.5, L, GRID_T_MAX, history_cap=L, precision=precision)
    hist = frozen_case(sv, 4097, L - 6, 9e6)
    grid = OI.Grid(L, GRID_T_MAX, 4)
    H = OI.History(*hist)
    model = Model(MIXED_34, 0.5)
    C, R = hist[1][-1], hist[3][-1]
    t_last = float(hist[0][-1])
    for t in (t_last, t_last * (1.0 + 1e-3)):
        S, mu = sv.history_integrals(t, C, R)
        assert np.all(np.isfinite(S))
        Sref = OI.history_integrals(model, grid, H, t, C, R, js=ROWS)
        err = np.max(np.abs(S[:, ROWS] - Sref[:, ROWS]))
        assert err < TOL[precision], (t, err)
    sv.close()


def _golden():
    if not os.path.exists(GOLDEN):
        pytest.fail("stored oracle solve missing: run tests/golden/make_mixed34_quench.py 4097")
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.mark.parametrize("precision", ["fp64", "df"])
def test_quench_on_L4097_grid_matches_oracle_step_by_step(precision):
    need_gpu()
    from paper_2604_06309_gb300 import Solver
    g = _golden()
    c = g["case"]
    cols = np.array(g["columns"])
    sv = Solver({int(p): q for p, q in c["coefs"].items()}, c["T"], c["L"], c["grid_t_max"], s=c["s"],
                history_cap=c["history_cap"], precision=precision)
    for cp in g["checkpoints"]:
        assert sv.integrate(cp["t"], c["tol"]) == 0
        tg, Cg, _, Rg, _ = sv.get_history()
        # identical step decisions: the same slice times and counters
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
