"""Helpers shared by the GPU parity tests (seeded inputs, oracle references)."""
import numpy as np
import pytest

from paper_2604_06309_gb300.inputs import geometric_times, synthetic_history


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    import os
    from paper_2604_06309_gb300 import dmfe
    if not os.path.exists(dmfe.LIB_PATH):
        __graft_entry__.build()
    return torch


def frozen_case(sv, seed, n_slices, t_last, t_first=1e-2):
    times = geometric_times(n_slices, t_first, t_last)
    C, dC, R, dR = synthetic_history(seed, times, sv.theta, sv.omega)
    sv.set_history(times, C, dC, R, dR)
    return times, C, dC, R, dR
