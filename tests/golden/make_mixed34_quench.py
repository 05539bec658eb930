"""Writes mixed34_T0.5_L<L>.json: the oracle's solve of the mixed (3+4)-spin quench
(f = (q^3 + q^4)/4, T = 0.5, random initial condition, Secs. 2.1 and 3.1-3.6) on one of
the benchmark grids, s = 4, a store of L slices, tolerance 1e-8, from t = 0:

  L = 2049 (grid t_max 1e5): states at t = 0.1 and t = 1 (241 and 464 steps);
  L = 4097 (grid t_max 1e7): states at t = 0.005 and t = 0.02 (a few dozen and ~110 steps).

Each state holds the slice times, counters, E, mu, every eighth column and the last 32
columns of the final C and R rows, and two-time values.

Only the oracle is called. Its history integrals are split over output rows between
worker processes (rows are independent; each row's sums are the oracle's own). Run from
the repository root (L = 2049: about an hour on 8 cores; L = 4097: about as long):
    python tests/golden/make_mixed34_quench.py L [workers]
"""
import json
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import integrals as OI  # noqa: E402
from oracle import solver as OS  # noqa: E402

CASES = {
    2049: (dict(coefs={3: 0.25, 4: 0.25}, T=0.5, L=2049, grid_t_max=1e5, s=4, history_cap=2049, tol=1e-8),
           [0.1, 1.0]),
    4097: (dict(coefs={3: 0.25, 4: 0.25}, T=0.5, L=4097, grid_t_max=1e7, s=4, history_cap=4097, tol=1e-8),
           [0.005, 0.02]),
}
PAIRS = [(1.0, 0.0), (1.0, 0.5), (1.0, 0.9), (1.0, 0.99), (0.8, 0.3), (0.6, 0.59), (0.5, 0.1),
         (0.3, 0.0), (0.9, 0.45), (0.75, 0.7)]

_serial = OI.history_integrals


def columns(L):
    return sorted(set(range(0, L, 8)) | set(range(L - 32, L)))


def _rows(args):
    model, grid, hist, t, C, R, js = args
    return js, _serial(model, grid, hist, t, C, R, js=js)[:, js]


def main():
    L = int(sys.argv[1])
    workers = int(sys.argv[2]) if len(sys.argv) > 2 else os.cpu_count()
    c, checkpoints = CASES[L]
    pool = mp.get_context("spawn").Pool(workers)

    def parallel(model, grid, hist, t, C, R, js=None, j_chunk=256):
        assert js is None
        parts = np.array_split(np.arange(grid.L), 4 * workers)
        S = np.zeros((OI.NS, grid.L))
        for js_, block in pool.imap_unordered(_rows, [(model, grid, hist, t, C, R, p) for p in parts]):
            S[:, js_] = block
        return S

    OI.history_integrals = parallel
    sv = OS.Solver(c["coefs"], c["T"], L=c["L"], grid_t_max=c["grid_t_max"], s=c["s"],
                   history_cap=c["history_cap"])
    cols = columns(c["L"])
    out = {"case": {k: (v if k != "coefs" else {str(p): q for p, q in v.items()}) for k, v in c.items()},
           "columns": cols, "checkpoints": []}
    for tc in checkpoints:
        st = sv.integrate(tc, c["tol"])
        assert st == OS.OK
        t = np.array([a * tc for a, _ in PAIRS])
        tp = np.array([b * tc for _, b in PAIRS])
        out["checkpoints"].append({
            "t": tc, "E": sv.E, "mu": sv.mu,
            "stats": {k: int(v) for k, v in sv.stats.items() if k != "max_eps_sparse"},
            "t_switch": sv.t_switch,
            "slice_times": sv.hist.t.tolist(),
            "C_cols": sv.hist.C[-1][cols].tolist(), "R_cols": sv.hist.R[-1][cols].tolist(),
            "pairs": [[a, b] for a, b in zip(t.tolist(), tp.tolist())],
            "C_pairs": sv.get_C(t, tp).tolist(), "R_pairs": sv.get_R(t, tp).tolist(),
        })
        print("t = %g: %d steps" % (tc, sv.stats["steps_accepted"]), flush=True)
    pool.close()
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mixed34_T0.5_L%d.json" % L)
    with open(path, "w") as f:
        json.dump(out, f, indent=0)
        f.write("\n")


if __name__ == "__main__":
    main()
