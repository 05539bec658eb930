"""Batched and continuously batched solves against the same solves run alone."""
import numpy as np
import pytest

from gpu_common import need_gpu
from paper_2604_06309_gb300.inputs import MIXED_34, PURE_3

pytestmark = pytest.mark.gpu

CASES = [  # (f, T, L, cap, grid t_max, t_max)
    (MIXED_34, 0.5, 33, 24, 100.0, 1.5),
    (PURE_3, 0.8, 65, 64, 100.0, 1.0),
    ({3: 0.4, 4: 0.1}, 0.3, 129, 48, 1e3, 0.7),
]


def _alone(case, precision, tol):
    from paper_2604_06309_gb300 import Solver
    f, T, L, cap, gtm, tmax = case
    sv = Solver(f, T, L, gtm, history_cap=cap, precision=precision)
    assert sv.integrate(tmax, tol) == 0
    out = sv.get_history()
    st = sv.stats()
    sv.close()
    return out, st


@pytest.mark.parametrize("precision", ["fp64", "df", "fp32"])
def test_batch_is_bitwise_equal_to_solo_runs(precision):
    need_gpu()
    from paper_2604_06309_gb300 import Batch
    tol = 1e-8
    b = Batch(8, 129, 64, precision=precision)
    slots = [b.add(f, T, L, gtm, tmax, tol, history_cap=cap) for (f, T, L, cap, gtm, tmax) in CASES]
    b.run()
    status, t, running = b.poll()
    assert running == 0
    for case, k in zip(CASES, slots):
        assert status[k] == 1 and t[k] == case[5]
        ref, st = _alone(case, precision, tol)
        got = b.solver(k).get_history()
        for x, y in zip(got, ref):
            assert np.array_equal(x, y)
        assert b.solver(k).stats()["sparsify_passes"] == st["sparsify_passes"]
    b.close()


def test_continuous_batching_admits_and_releases_between_steps():
    """A request admitted while others run, and a slot reused after release, give the
    same result as running alone."""
    need_gpu()
    from paper_2604_06309_gb300 import Batch
    tol = 1e-8
    b = Batch(2, 129, 64, precision="df")

    def admit(c):
        f, T, L, cap, gtm, tmax = c
        return b.add(f, T, L, gtm, tmax, tol, history_cap=cap)

    admit(CASES[0])
    b.step(40)
    admit(CASES[1])          # joins while the first solve is running
    pending = [CASES[2]]     # waits for a free slot
    results = {}
    for _ in range(10000):
        b.step(8)
        status, t, running = b.poll()
        assert not any(-100 < s_ < 0 for s_ in status)
        for k in range(2):
            if status[k] == 1:
                sv = b.solver(k)
                results[sv.L] = sv.get_history()
                b.remove(k)
                if pending:
                    admit(pending.pop())
        if len(results) == len(CASES):
            break
    assert len(results) == len(CASES)
    for case in CASES:
        ref, _ = _alone(case, "df", tol)
        for x, y in zip(results[case[2]], ref):
            assert np.array_equal(x, y)
    b.close()
