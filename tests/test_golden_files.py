"""The stored oracle solves under tests/golden/ against the oracle as it stands (the first
checkpoint is recomputed where that takes seconds) and against properties every solve of
the DMFE has (Secs. 2.1 and 3.1): C(t, t) = R(t, t-) = 1, |C| <= 1, causality of the
stored slices, mu = T - p E for a pure p-spin model with f = q^p / 2."""
import json
import os

import numpy as np
import pytest

from oracle import solver as OS

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FILES = ["pure3_T0.8_L129.json", "mixed34_T0.5_L2049.json", "mixed34_T0.5_L4097.json"]


def _load(name):
    path = os.path.join(HERE, name)
    if not os.path.exists(path):
        pytest.skip("%s not written" % name)
    with open(path) as f:
        return json.load(f)


@pytest.mark.parametrize("name", FILES)
def test_stored_solves_have_the_invariants(name):
    g = _load(name)
    c = g["case"]
    for cp in g["checkpoints"]:
        ts = np.array(cp["slice_times"])
        assert ts[0] == 0.0 and np.all(np.diff(ts) > 0) and abs(ts[-1] - cp["t"]) < 1e-12 * cp["t"]
        C = np.array(cp.get("C_row", cp.get("C_cols")))
        R = np.array(cp.get("R_row", cp.get("R_cols")))
        # the last stored column is theta = 1: the equal-time values
        assert C[-1] == 1.0 and R[-1] == 1.0
        assert np.all(np.abs(C) <= 1.0 + 1e-12)
        pairs = np.array(cp["pairs"])
        Cp, Rp = np.array(cp["C_pairs"]), np.array(cp["R_pairs"])
        eq = pairs[:, 0] == pairs[:, 1]
        assert np.all(np.abs(Cp[eq] - 1.0) < 1e-12)
        assert np.all(np.abs(Cp) <= 1.0 + 1e-12) and np.all(np.isfinite(Rp))
        coefs = {int(p): q for p, q in c["coefs"].items()}
        if len(coefs) == 1:
            p, q = next(iter(coefs.items()))
            if q == 0.5:
                assert abs(cp["mu"] - (c["T"] - p * cp["E"])) < 1e-8


@pytest.mark.parametrize("name", ["mixed34_T0.5_L2049.json", "mixed34_T0.5_L4097.json"])
def test_early_steps_follow_the_step_rule(name):
    """Sec. 3.5 step rule (reading R7): from dt0 = 1e-4 an accepted step with eps_RK < tol/2
    multiplies dt by 1.01, and the last step is shortened to land on the target. Before the
    first checkpoint of the benchmark-grid quenches nothing is rejected or removed, so the
    stored slice times are the partial sums 1e-4 (1.01^k - 1) / 0.01."""
    g = _load(name)
    cp = g["checkpoints"][0]
    st = cp["stats"]
    assert st["steps_rejected"] == 0 and st["slices_removed"] == 0
    ts = np.array(cp["slice_times"])
    k = np.arange(len(ts) - 1)
    expect = 1e-4 * (1.01 ** k - 1.0) / 0.01
    assert len(ts) == st["steps_accepted"] + 1
    assert np.max(np.abs(ts[:-1] - expect) / np.maximum(expect, 1e-300)) < 1e-13
    assert ts[-1] == cp["t"] and ts[-1] - ts[-2] <= 1e-4 * 1.01 ** (len(ts) - 2) * (1 + 1e-13)


def test_small_quench_first_checkpoint_reproduces():
    """The oracle as it stands reproduces the stored L = 129 solve to t = 1 exactly."""
    g = _load("pure3_T0.8_L129.json")
    c = g["case"]
    cp = g["checkpoints"][0]
    sv = OS.Solver({int(p): q for p, q in c["coefs"].items()}, c["T"], L=c["L"], grid_t_max=c["grid_t_max"],
                   history_cap=c["history_cap"])
    assert sv.integrate(cp["t"], c["tol"]) == OS.OK
    assert np.array_equal(sv.hist.t, np.array(cp["slice_times"]))
    assert np.max(np.abs(sv.hist.C[-1] - np.array(cp["C_row"]))) < 1e-13
    assert np.max(np.abs(sv.hist.R[-1] - np.array(cp["R_row"]))) < 1e-13
    assert abs(sv.E - cp["E"]) < 1e-13
