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


def _alone(case, precision, tol, hi_chunk=0):
    from paper_2604_06309_gb300 import Solver
    f, T, L, cap, gtm, tmax = case
    # a batch slot runs one work unit per output index (hi_chunk = L) unless given a unit
    # size: the same here, so that the summation order, and hence every bit, agrees
    sv = Solver(f, T, L, gtm, history_cap=cap, precision=precision, hi_chunk=hi_chunk or L)
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


@pytest.mark.parametrize("precision", ["fp64", "df"])
def test_autotuned_units_keep_batch_equal_to_solo_runs(precision):
    """The batch autotuner's choice, given to a fresh batch, keeps every slot bitwise equal
    to the same solve run alone with that unit size."""
    need_gpu()
    from paper_2604_06309_gb300 import Batch
    tol = 1e-8
    a = Batch(8, 129, 64, precision=precision)
    for (f, T, L, cap, gtm, tmax) in CASES:
        a.add(f, T, L, gtm, tmax, tol, history_cap=cap)
    a.step(20)
    chunk, ms = a.autotune(2)
    a.close()
    assert chunk in ms and all(v > 0 for v in ms.values())
    b = Batch(8, 129, 64, precision=precision)
    slots = [b.add(f, T, L, gtm, tmax, tol, history_cap=cap, hi_chunk=chunk) for (f, T, L, cap, gtm, tmax) in CASES]
    b.run()
    for case, k in zip(CASES, slots):
        ref, st = _alone(case, precision, tol, hi_chunk=chunk)
        got = b.solver(k).get_history()
        for x, y in zip(got, ref):
            assert np.array_equal(x, y)
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


def _wait_results(srv, n, timeout=120.0):
    import time
    res = {}
    t0 = time.time()
    while len(res) < n and time.time() - t0 < timeout:
        for r in srv.poll():
            res[r["id"]] = r
        time.sleep(0.005)
    return res


def test_server_results_equal_solo_runs():
    need_gpu()
    from paper_2604_06309_gb300 import Server, Solver
    tol = 1e-8
    srv = Server(4, 129, 64, precision="df", hbm_budget=8 << 30, steps_per_round=4)
    ids = {}
    for c in CASES:
        f, T, L, cap, gtm, tmax = c
        ids[srv.submit(f, T, L, gtm, tmax, tol, history_cap=cap)] = c
    res = _wait_results(srv, len(CASES))
    st = srv.stats()
    srv.stop()
    assert len(res) == len(CASES) and st["completed"] == len(CASES) and st["failed"] == 0
    for rid, c in ids.items():
        f, T, L, cap, gtm, tmax = c
        sv = Solver(f, T, L, gtm, history_cap=cap, precision="df", hi_chunk=L)
        assert sv.integrate(tmax, tol) == 0
        t, _, _, mu, E = sv.get_row()
        r = res[rid]
        assert r["status"] == 0 and r["t_final"] == t and r["E"] == E and r["mu"] == mu
        assert r["submit_s"] <= r["admit_s"] <= r["done_s"]
        sv.close()


def test_server_admission_respects_the_footprint_budget():
    need_gpu()
    import time
    from paper_2604_06309_gb300 import Server, footprint
    c = CASES[2]
    f, T, L, cap, gtm, tmax = c
    one = footprint(f, T, L, gtm, history_cap=cap, precision="fp64")
    srv = Server(4, 129, 64, precision="fp64", hbm_budget=int(1.5 * one), steps_per_round=2)
    ids = [srv.submit(f, T, L, gtm, tmax, 1e-8, history_cap=cap) for _ in range(3)]
    seen = 0
    res = {}
    t0 = time.time()
    while len(res) < 3 and time.time() - t0 < 120:
        st = srv.stats()
        seen = max(seen, st["running"])
        assert st["bytes_in_use"] <= int(1.5 * one)
        for r in srv.poll():
            res[r["id"]] = r
        time.sleep(0.002)
    srv.stop()
    assert len(res) == 3 and seen == 1
    # later requests waited for the earlier ones
    order = sorted(res.values(), key=lambda r: r["admit_s"])
    assert order[1]["admit_s"] >= order[0]["done_s"] - 1e-3
    with pytest.raises(Exception):
        Server(1, 129, 64, hbm_budget=one // 2).submit(f, T, L, gtm, tmax, 1e-8, history_cap=cap)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "df"])
def test_footprint_covers_the_allocations(precision):
    torch = need_gpu()
    from paper_2604_06309_gb300 import Solver, footprint
    L, cap = 1025, 600
    est = footprint(MIXED_34, 0.5, L, 1e4, history_cap=cap, precision=precision)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    sv = Solver(MIXED_34, 0.5, L, 1e4, history_cap=cap, precision=precision)
    free1, _ = torch.cuda.mem_get_info()
    used = free0 - free1
    sv.close()
    assert used <= est * 1.02 + (8 << 20)
    assert est <= used * 1.25 + (64 << 20)
