"""The allocation-free sparsification entry point against the solver's dmfe_sparsify.

dmfe_sparsify_select_noalloc is for callers that cannot call cudaMalloc (their device
memory belongs to another framework's pool, or they cannot afford an allocation's
synchronisation) and so cannot create a solver. It must give the same removal decision
as the existing entry point. Two calls in a row, the second on a smaller history, check
that the shared fixed scratch array carries nothing over from one call to the next.
This file is collected last so that a failure here does not hide the other tests.
"""
import ctypes

import numpy as np
import pytest

from gpu_common import need_gpu
from paper_2604_06309_gb300.inputs import MIXED_34, synthetic_history

pytestmark = pytest.mark.gpu


def _history(L, seed, n_dense):
    from paper_2604_06309_gb300 import Solver
    g = Solver(MIXED_34, 0.5, L, 1e3, history_cap=16)  # only for the theta grid
    th, om = g.theta.copy(), g.omega.copy()
    g.close()
    times = np.concatenate([[0.0], np.geomspace(1e-2, 50.0, 60), np.linspace(50.5, 60.0, n_dense)])
    return (times,) + synthetic_history(seed, times, th, om)


def _existing_entry(L, hist, tol):
    from paper_2604_06309_gb300 import Solver
    sv = Solver(MIXED_34, 0.5, L, 1e3, history_cap=max(16, len(hist[0])))
    sv.set_history(*hist)
    removed = sv.sparsify(tol)
    sv.close()
    return removed


def _noalloc_entry(torch, lib, L, hist, tol):
    t, C, dC, R, dR = (torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda") for a in hist)
    n = t.numel()
    out = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    rc = lib.dmfe_sparsify_select_noalloc(t.data_ptr(), C.data_ptr(), dC.data_ptr(), R.data_ptr(),
                                          dR.data_ptr(), n, L, tol, out.data_ptr(), stream.cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(bool)


def test_noalloc_matches_dmfe_sparsify_on_two_calls_in_a_row():
    torch = need_gpu()
    from paper_2604_06309_gb300 import dmfe
    lib = dmfe.load()
    L, tol = 65, 1e-8
    first = _history(L, 31, 179)    # 240 slices
    second = _history(L, 32, 40)    # 101 slices: a shorter call after a longer one
    for hist in (first, second):
        expect = _existing_entry(L, hist, tol)
        got = _noalloc_entry(torch, lib, L, hist, tol)
        assert got.shape == expect.shape
        assert np.array_equal(got, expect)
        assert 0 < got.sum() < len(got)


def test_noalloc_forced_removal_and_short_history_match_dmfe_sparsify():
    """Two branches the greedy rule does not reach: with tol = 1e-30 no residual
    qualifies and both entries force-remove the candidate with the smallest residual;
    with n <= 12 slices there are no candidates and both remove nothing."""
    torch = need_gpu()
    from paper_2604_06309_gb300 import dmfe
    lib = dmfe.load()
    L = 65
    hist = _history(L, 33, 60)      # 121 slices
    expect = _existing_entry(L, hist, 1e-30)
    got = _noalloc_entry(torch, lib, L, hist, 1e-30)
    assert np.array_equal(got, expect)
    assert got.sum() == 1 and 1 <= int(np.argmax(got)) <= len(got) - 12
    short = tuple(a[:12] for a in _history(L, 34, 0))
    expect = _existing_entry(L, short, 1e-8)
    got = _noalloc_entry(torch, lib, L, short, 1e-8)
    assert np.array_equal(got, expect) and got.sum() == 0


def test_noalloc_rejects_sizes_beyond_its_fixed_scratch():
    torch = need_gpu()
    from paper_2604_06309_gb300 import dmfe
    lib = dmfe.load()
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = torch.zeros(16, dtype=torch.int32, device="cuda")
    p = buf.data_ptr()
    rc = lib.dmfe_sparsify_select_noalloc(p, p, p, p, p, 16384 + 1, 1, 1e-8, out.data_ptr(), None)
    assert rc == dmfe.DMFE_ERR_ARG
