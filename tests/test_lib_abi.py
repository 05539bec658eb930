"""CPU checks of the C ABI: the library loads, exports every declared symbol and the
ctypes structures match the C layout (no GPU work)."""
import ctypes
import os
import re
import subprocess

import numpy as np
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
                    ' offsetof(dmfe_params, stream), offsetof(dmfe_stats_t, status), offsetof(dmfe_stats_t, precision));'
                    'printf("%zu %zu\\n", offsetof(dmfe_params, sparsify_every), offsetof(dmfe_params, sparsify_passes));'
                    'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    vals = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert vals == [ctypes.sizeof(dmfe.dmfe_params), ctypes.sizeof(dmfe.dmfe_stats_t),
                    dmfe.dmfe_params.stream.offset, dmfe.dmfe_stats_t.status.offset,
                    dmfe.dmfe_stats_t.precision.offset, dmfe.dmfe_params.sparsify_every.offset,
                    dmfe.dmfe_params.sparsify_passes.offset]


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


def test_every_field_offset_matches_c(tmp_path):
    """Offsets of every field of the four public structures, C against ctypes."""
    from paper_2604_06309_gb300 import dmfe
    structs = [("dmfe_params", dmfe.dmfe_params), ("dmfe_stats_t", dmfe.dmfe_stats_t),
               ("dmfe_result", dmfe.dmfe_result), ("dmfe_server_stats_t", dmfe.dmfe_server_stats_t)]
    lines = []
    for cname, ct in structs:
        lines.append('printf("%%zu\\n", sizeof(%s));' % cname)
        for f, _ in ct._fields_:
            lines.append('printf("%%zu\\n", offsetof(%s, %s));' % (cname, f))
    prog = tmp_path / "off.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "dmfe.h"\nint main(void){%s return 0;}\n'
                    % "".join(lines))
    exe = tmp_path / "off"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = []
    for _, ct in structs:
        want.append(ctypes.sizeof(ct))
        want += [getattr(ct, f).offset for f, _ in ct._fields_]
    assert got == want


def test_defaults_and_host_side_validation_without_gpu(built):
    """dmfe_default_params, dmfe_footprint and the parameter checks of dmfe_create run on
    the host only (no device call happens before a parameter is rejected)."""
    from paper_2604_06309_gb300 import dmfe
    lib = dmfe.load()
    p = dmfe.dmfe_params()
    lib.dmfe_default_params(ctypes.byref(p))
    assert (p.L, p.s, p.precision, p.sparsify, p.integrator, p.rk_switch_dt, p.hi_chunk, p.interp, p.fh_d,
            p.log_r) == (513, 4, 0, 1, 0, 0.0, 0, 0, 3, 0)
    assert p.dt0 == 1e-4 and p.dt_min == 1e-12 and p.grid_t_max == 1e5

    def params(**kw):
        prm, keep = dmfe.make_params({3: 0.25, 4: 0.25}, 0.5, kw.pop("L", 129), kw.pop("grid_t_max", 1e3), **kw)
        return prm, keep

    # footprint: grows with L and the store; FP64 (weight tables, interval coefficients) >
    # double-float (positions, replica) > FP32 (packed positions, FP32 replica)
    fp = lambda **kw: lib.dmfe_footprint(ctypes.byref(params(**kw)[0]))
    assert fp(L=257) > fp(L=129) > 0
    assert fp(L=129, history_cap=400) > fp(L=129)
    assert fp(precision="fp64") > fp(precision="df") > fp(precision="fp32")
    # log-R mode: one table of four log-R coefficients per stored interval and buffer
    # (history_cap defaults to L; allocations are counted in 512-byte granules)
    assert 0 <= fp(log_r=True) - fp() - 2 * 129 * 129 * 32 < 2 * 512
    h = ctypes.c_void_p()
    bad = [dict(L=8), dict(s=5), dict(history_cap=8), dict(dt0=0.0), dict(hi_chunk=16), dict(fh_d=4, interp="fh_index")]
    for kw in bad:
        prm, keep = params(**kw)
        rc = lib.dmfe_create(ctypes.byref(prm), ctypes.byref(h))
        assert rc in (-1, -8), (kw, rc)
        assert fp(**kw) == 0 if rc == -1 else True
    for prec in ("df", "fp32"):          # the rational and theta-space stencils need FP64
        prm, keep = params(precision=prec, interp="fh_index")
        assert lib.dmfe_create(ctypes.byref(prm), ctypes.byref(h)) == -8
        prm, keep = params(precision=prec, log_r=True)   # so does the log-R interpolation
        assert lib.dmfe_create(ctypes.byref(prm), ctypes.byref(h)) == -8
    prm, keep = params()
    prm.log_r = 2
    assert lib.dmfe_create(ctypes.byref(prm), ctypes.byref(h)) == -1
    prm, keep = params()
    prm.integrator = 7
    assert lib.dmfe_create(ctypes.byref(prm), ctypes.byref(h)) == -1
    prm, keep = params(grid_t_max=2.0)   # gamma = -W_{-1}(-1/t_max) needs t_max > e
    assert lib.dmfe_create(ctypes.byref(prm), ctypes.byref(h)) == -1


@pytest.mark.parametrize("L,t_max,alpha,delta", [(33, 10.0, 0.0, 0.0), (129, 100.0, 0.0, 0.0),
                                                  (257, 1e4, 0.5, 0.2), (2049, 1e5, 0.0, 0.0),
                                                  (4097, 1e7, 0.0, 0.0)])
def test_host_grid_matches_oracle_without_gpu(built, L, t_max, alpha, delta):
    """The library's host code for Eq. (theta) and the weights of Sec. 3.4 (the grid every
    solver is built on), called through dmfe_theta_grid on the CPU, against the oracle."""
    from oracle import grid as og, quadrature as oq
    from paper_2604_06309_gb300 import theta_grid
    th, om, nu = theta_grid(L, t_max, alpha, delta)
    ref_th, ref_om = og.theta_grid(L, og.gamma_from_tmax(t_max), alpha, delta)
    # numpy's and the C library's exp/atan may differ by an ulp or two; theta takes a few
    # of them through the quotient of Eq. (theta)
    assert np.max(np.abs(th - ref_th)) < 2e-15
    assert np.max(np.abs(om - ref_om) / np.maximum(ref_om, 1e-300)) < 1e-14
    ref_nu = oq.spline_weights(ref_th)
    assert np.max(np.abs(nu - ref_nu)) < 1e-13 * max(1.0, np.max(np.abs(ref_nu)) * L)


def test_host_grid_rejects_bad_arguments(built):
    from paper_2604_06309_gb300 import DMFEError, theta_grid
    for args in [(8, 100.0), (129, 2.0), (129, 100.0, 1.5), (129, 100.0, 0.0, -1.0)]:
        with pytest.raises(DMFEError) as e:
            theta_grid(*args)
        assert e.value.code == -1

