"""The bounds-checked build (libdmfe_checked.so, -DDMFE_CHECKED): every stencil base and
history row index of the history-integral and sparsification kernels is tested before its
access, and a failure is recorded in the solver's bounds_site word instead of trapping.
On valid inputs no check may fail and the results must equal the normal build's bit for
bit. The checked cases run in a child process (the library is chosen at load time)."""
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_common import need_gpu

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_reports_no_failure_and_matches_normal_build(tmp_path):
    need_gpu()
    from paper_2604_06309_gb300 import build as B, dmfe
    if not os.path.exists(dmfe.CHECKED_LIB_PATH):
        B.build(checked=True)
    import checked_case
    normal = checked_case.run()
    out = tmp_path / "checked.npz"
    env = dict(os.environ, DMFE_LIBRARY=dmfe.CHECKED_LIB_PATH)
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_case.py"), str(out)], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    checked = np.load(out)
    assert sorted(checked.files) == sorted(normal)
    for k in normal:
        if k.endswith("_bounds"):
            assert int(checked[k]) == 0 and int(normal[k]) == 0, k
        else:
            assert np.array_equal(checked[k], normal[k]), k
