"""Cases run once with the normal library and once with the bounds-checked build
(libdmfe_checked.so, selected by DMFE_LIBRARY in a child process) by
tests/test_gpu_checked.py. Every output array and every solver's bounds_site word is
collected into one dict.

    python tests/checked_case.py OUT.npz      (runs with whatever DMFE_LIBRARY selects)
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def run():
    from paper_2604_06309_gb300 import Batch, Solver
    from paper_2604_06309_gb300.inputs import MIXED_34, PURE_3, geometric_times, synthetic_history
    out = {}

    def frozen(tag, L, s, n, t_last, precision, log_r=False):
        sv = Solver(MIXED_34, 0.5, L, 1e5, s=s, history_cap=max(n, 16), precision=precision, log_r=log_r)
        times = geometric_times(n, 1e-2, t_last)
        C, dC, R, dR = synthetic_history(L + n, times, sv.theta, sv.omega)
        if log_r:
            R = np.abs(R) + 1e-3  # positive responses: the logarithmic reads are taken
        sv.set_history(times, C, dC, R, dR)
        for k, t in enumerate((times[-1], times[-1] * 1.001)):
            out["%s_S%d" % (tag, k)] = sv.history_integrals(t, C[-1], R[-1])[0]
        out[tag + "_bounds"] = np.array(sv.stats()["bounds_site"])
        sv.close()

    for prec in ("fp64", "df", "fp32"):
        frozen("frozen129_%s" % prec, 129, 4, 130, 300.0, prec)
        frozen("frozen129s10_%s" % prec, 129, 10, 60, 300.0, prec)
        frozen("frozen2049_%s" % prec, 2049, 4, 2043, 9e4, prec)
    frozen("frozen257_logr", 257, 4, 200, 500.0, "fp64", log_r=True)

    def solve(tag, precision, **kw):
        sv = Solver(MIXED_34, 0.5, 33, 100.0, history_cap=24, dt0=0.3, precision=precision, **kw)
        rc = sv.integrate(2.0, 1e-8)
        t, C, dC, R, dR = sv.get_history()
        st = sv.stats()
        out[tag + "_hist"] = np.concatenate([t[:, None], C, dC, R, dR], axis=1)
        out[tag + "_counts"] = np.array([rc, st["steps_accepted"], st["steps_rejected"], st["sparsify_passes"],
                                         st["slices_removed"], st["forced_removals"]])
        out[tag + "_bounds"] = np.array(st["bounds_site"])
        sv.close()

    for prec in ("fp64", "df", "fp32"):
        solve("solve_%s" % prec, prec)
    solve("solve_ssprk_passes", "fp64", integrator="ssprk104", sparsify_every=3, sparsify_passes=2)

    for prec in ("fp64", "df"):
        b = Batch(4, 65, 64, precision=prec)
        slots = [b.add(coefs, T, L, 100.0, 1.0, 1e-8, history_cap=32 + 8 * k)
                 for k, (coefs, T, L) in enumerate(((MIXED_34, 0.5, 33), (PURE_3, 0.8, 65), (MIXED_34, 0.7, 65),
                                                    (PURE_3, 0.6, 33)))]
        b.step(120)
        b.poll()
        for k, slot in enumerate(slots):
            sv = b.solver(slot)
            t, C, dC, R, dR = sv.get_history()
            out["batch_%s_%d_hist" % (prec, k)] = np.concatenate([t[:, None], C, dC, R, dR], axis=1)
            out["batch_%s_%d_bounds" % (prec, k)] = np.array(sv.stats()["bounds_site"])
        b.close()
    return out


if __name__ == "__main__":
    import torch
    torch.cuda.set_device(0)
    np.savez(sys.argv[1], **run())
