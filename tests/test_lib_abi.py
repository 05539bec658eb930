"""CPU checks of the C ABI: the library loads, exports every declared symbol and the
ctypes structures match the C layout (no GPU work)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "include", "dmfe.h")
LIB = os.path.join(ROOT, "paper_2604_06309_gb300", "libdmfe.so")


@pytest.fixture(scope="module")
def built():
    if not os.path.exists(LIB):
        from paper_2604_06309_gb300.build import build
        build()
    return LIB


def declared_functions():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dmfe_[A-Za-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(built):
    lib = ctypes.CDLL(built)
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_binding_declares_every_symbol():
    from paper_2604_06309_gb300 import dmfe
    assert sorted(dmfe._SIGS) == declared_functions()


def test_struct_layout_matches_c(tmp_path):
    from paper_2604_06309_gb300 import dmfe
    prog = tmp_path / "sz.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "dmfe.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu\\n", sizeof(dmfe_params), sizeof(dmfe_stats_t),'
                    ' offsetof(dmfe_params, stream), offsetof(dmfe_stats_t, status), offsetof(dmfe_stats_t, precision));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    vals = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert vals == [ctypes.sizeof(dmfe.dmfe_params), ctypes.sizeof(dmfe.dmfe_stats_t),
                    dmfe.dmfe_params.stream.offset, dmfe.dmfe_stats_t.status.offset,
                    dmfe.dmfe_stats_t.precision.offset]


def test_strerror_without_gpu(built):
    from paper_2604_06309_gb300 import dmfe
    lib = dmfe.load()
    assert lib.dmfe_strerror(-4) == b"step size fell below dt_min"
    assert lib.dmfe_strerror(0) == b"ok"


def test_create_rejects_bad_arguments_before_touching_the_gpu(built):
    from paper_2604_06309_gb300 import dmfe
    lib = dmfe.load()
    p = dmfe.dmfe_params()
    lib.dmfe_default_params(ctypes.byref(p))
    h = ctypes.c_void_p()
    assert lib.dmfe_create(ctypes.byref(p), ctypes.byref(h)) == dmfe.DMFE_ERR_ARG  # no f given
    pw = (ctypes.c_int * 1)(3)
    cf = (ctypes.c_double * 1)(0.5)
    p.n_terms, p.powers, p.coefs = 1, ctypes.cast(pw, dmfe._ip), ctypes.cast(cf, dmfe._dp)
    p.s = 5
    assert lib.dmfe_create(ctypes.byref(p), ctypes.byref(h)) == dmfe.DMFE_ERR_UNSUPPORTED
    p.s = 4
    p.grid_t_max = 2.0
    assert lib.dmfe_create(ctypes.byref(p), ctypes.byref(h)) == dmfe.DMFE_ERR_ARG
    assert not h.value
