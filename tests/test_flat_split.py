"""The flat split's host tables on CPU (tests/flat_split_check.cu, built with nvcc for the
host only): for grids L = 512 .. 4097 and warp counts from full launches of 152 SMs x 16
warps down to a single warp, every pair is covered once, every row's parts arrive in
order, and no row has more parts than the partial-sum buffer holds; the fit rule refuses
grids below L = 512 and segments under 256 pairs."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _fits(L, G):
    return G > 0 and L * L >= 256 * G and L >= 512


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path_factory.mktemp("flat") / "flat_split_check"
    subprocess.check_call([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                           "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "flat_split_check.cu"),
                           "-o", str(exe)])
    return str(exe)


def test_tables_cover_every_pair_once_in_part_order(checker):
    cases = []
    for L in (512, 513, 777, 1025, 2049, 4097):
        for G in (152 * 16, 152 * 8, 148 * 16, 132 * 16, 152 * 12, 1000, 99, 7, 1, L * L // 256):
            if _fits(L, G):
                cases += [L, G]
    out = subprocess.run([checker] + [str(x) for x in cases], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip() == "ok %d" % (len(cases) // 2)


def test_fit_rule_refuses_small_grids_and_short_segments(checker):
    for L, G in ((511, 1), (256, 4), (512, 1025), (1024, 4097)):
        assert not _fits(L, G)
        out = subprocess.run([checker, str(L), str(G)], capture_output=True, text=True)
        assert out.returncode == 1 and "does not fit" in out.stdout
