"""The C ABI library loads and exports every symbol include/scgal.h declares
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "scgal.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(scgal_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1912_02949_gb300 import build, scgal
    build.build()
    return scgal.load()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("scgal_create_maxcut", "scgal_create_phase", "scgal_step", "scgal_solve",
                 "scgal_reconstruct", "scgal_submit", "scgal_poll", "scgal_destroy", "scgal_strerror"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_exactly_the_header():
    from paper_1912_02949_gb300 import scgal
    assert sorted(scgal._PROTOS) == _declared()


def test_struct_layouts_match_c(lib):
    """Compile a C program against the header and compare sizes and offsets."""
    from paper_1912_02949_gb300 import scgal as S
    structs = {"scgal_params": S.scgal_params, "scgal_stats": S.scgal_stats, "scgal_info": S.scgal_info,
               "scgal_result": S.scgal_result, "scgal_server_stats": S.scgal_server_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "scgal.h"', "int main(void){"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(src, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(l.split() for l in out if l)
    for cname, py in structs.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, (cname, f)


def test_host_side_argument_checks_need_no_gpu(lib):
    from paper_1912_02949_gb300 import scgal as S
    p = S.scgal_params_default()
    assert (p.R, p.T_max, p.precision, p.scale, p.check_every) == (10, 1000, 32, 1, 16)
    h = ctypes.c_void_p()
    # n < 2 is rejected before any CUDA call
    assert lib.scgal_create_maxcut(None, None, None, 1, 0, 0.0, ctypes.byref(p), ctypes.byref(h)) == S.SCGAL_EINVAL
    bad = S.scgal_params_default(R=0)
    assert lib.scgal_create_phase(None, 12, 64, None, 0.0, ctypes.byref(bad), ctypes.byref(h)) == S.SCGAL_EINVAL
    # a sketch rank above n is rejected before any CUDA call
    rp = (ctypes.c_int32 * 3)(0, 1, 2)
    cl = (ctypes.c_int32 * 2)(1, 0)
    big = S.scgal_params_default(R=3)
    assert lib.scgal_create_maxcut(rp, cl, None, 2, 2, 0.0, ctypes.byref(big), ctypes.byref(h)) == S.SCGAL_EINVAL
    # an unknown test-matrix mode likewise
    assert S.scgal_params_default().omega == S.SCGAL_OMEGA_STORED
    ok = S.scgal_params_default(R=2, omega=2)
    assert lib.scgal_create_maxcut(rp, cl, None, 2, 2, 0.0, ctypes.byref(ok), ctypes.byref(h)) == S.SCGAL_EINVAL
    # and an unknown constraint set
    assert S.scgal_params_default().kset == S.SCGAL_K_EQ
    ok = S.scgal_params_default(R=2, kset=2)
    assert lib.scgal_create_maxcut(rp, cl, None, 2, 2, 0.0, ctypes.byref(ok), ctypes.byref(h)) == S.SCGAL_EINVAL
    m = (ctypes.c_double * 64)()
    big = S.scgal_params_default(R=17)
    assert lib.scgal_create_phase(m, 1, 16, m, 0.0, ctypes.byref(big), ctypes.byref(h)) == S.SCGAL_EINVAL
    # ptychography geometry is checked before any CUDA call: M a power of two in
    # [2, 64], s | N, M <= N
    pp = (ctypes.c_double * 128)()
    good = S.scgal_params_default(R=2)
    for (M, N, s_) in ((6, 12, 3), (8, 12, 5), (16, 8, 2), (128, 256, 2), (1, 4, 2)):
        assert lib.scgal_create_ptycho(pp, M, N, s_, pp, 0.0, ctypes.byref(good), ctypes.byref(h)) == S.SCGAL_EINVAL
    # a phase-retrieval submission without a server is rejected on the host
    t = ctypes.c_uint64()
    assert lib.scgal_submit_phase(None, pp, 1, 16, pp, ctypes.byref(good), ctypes.byref(t)) == S.SCGAL_EINVAL
    assert lib.scgal_strerror(S.SCGAL_ENUMERIC).decode() == "numerical failure"
    assert lib.scgal_step(None, None) == S.SCGAL_EINVAL
