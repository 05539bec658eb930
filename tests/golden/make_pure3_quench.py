"""Writes pure3_T0.8_L129.json: the oracle's solve of the pure 3-spin quench (f = q^3/2,
T = 0.8 above T_d, random initial condition, Secs. 2.1 and 3.1-3.6) on an L = 129 grid with
a 129-slice store, tolerance 1e-8, to t = 100, with the state at t = 1, 10 and 100.

Only the oracle is called. Run from the repository root:
    python tests/golden/make_pure3_quench.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import solver as OS  # noqa: E402

CASE = dict(coefs={3: 0.5}, T=0.8, L=129, grid_t_max=100.0, history_cap=129, tol=1e-8)
CHECKPOINTS = [1.0, 10.0, 100.0]
# two-time sample points (t, t') at each checkpoint, as fractions (t/t_c, t'/t_c)
PAIRS = [(1.0, 0.0), (1.0, 0.5), (1.0, 0.9), (1.0, 0.99), (0.8, 0.3), (0.6, 0.59), (0.5, 0.1),
         (0.3, 0.0), (0.9, 0.45), (0.75, 0.7)]


def main():
    c = CASE
    sv = OS.Solver(c["coefs"], c["T"], L=c["L"], grid_t_max=c["grid_t_max"], history_cap=c["history_cap"])
    out = {"case": {k: (v if k != "coefs" else {str(p): q for p, q in v.items()}) for k, v in c.items()},
           "checkpoints": []}
    for tc in CHECKPOINTS:
        st = sv.integrate(tc, c["tol"])
        assert st == OS.OK
        t = np.array([a * tc for a, _ in PAIRS])
        tp = np.array([b * tc for _, b in PAIRS])
        out["checkpoints"].append({
            "t": tc, "E": sv.E, "mu": sv.mu,
            "stats": {k: int(v) for k, v in sv.stats.items() if k != "max_eps_sparse"},
            "t_switch": sv.t_switch,
            "slice_times": sv.hist.t.tolist(),
            "C_row": sv.hist.C[-1].tolist(), "R_row": sv.hist.R[-1].tolist(),
            "pairs": [[a, b] for a, b in zip(t.tolist(), tp.tolist())],
            "C_pairs": sv.get_C(t, tp).tolist(), "R_pairs": sv.get_R(t, tp).tolist(),
        })
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "pure3_T0.8_L129.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=0)
        f.write("\n")


if __name__ == "__main__":
    main()
