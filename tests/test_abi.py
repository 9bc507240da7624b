"""Host-side checks of the C ABI (no GPU needed): libgmt.so loads, exports every
function include/gmt.h declares, and the ctypes structs have the C layout."""
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gmt.h")


@pytest.fixture(scope="module")
def native():
    from paper_1705_02403_gb300 import build
    build.build()
    from paper_1705_02403_gb300 import _native
    return _native


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gmt_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_function(native):
    names = declared_functions()
    assert names, "no declarations parsed"
    out = subprocess.run(["nm", "-D", "--defined-only", native.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s+(gmt_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    assert set(names) == set(native.SIGNATURES), "binding and header disagree"


def test_struct_layout_matches_c(native):
    import ctypes as C
    structs = ["gmt_space", "gmt_boxes", "gmt_goal", "gmt_params", "gmt_graph_view", "gmt_plan_info", "gmt_profile",
               "gmt_query", "gmt_model_config", "gmt_model_view", "gmt_server_config", "gmt_server_result"]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gmt.h"', "int main(void){"]
    for s in structs:
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f, _ in getattr(native, s)._fields_:
            cf = "lambda" if f == "lambda_" else f
            lines.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {cf}));')
    lines.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "layout.c")
        open(c, "w").write("\n".join(lines))
        exe = os.path.join(d, "layout")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(l.split() for l in out if l.strip())
    for s in structs:
        cls = getattr(native, s)
        assert int(got[s]) == C.sizeof(cls), s
        for f, _ in cls._fields_:
            assert int(got[f"{s}.{f}"]) == getattr(cls, f).offset, f"{s}.{f}"


def test_host_radius_matches_oracle(native, O):
    # Theorem 1's radius is computed on the host by both sides; equal doubles
    # give equal FP32 radii, hence equal graphs.
    for d in (2, 3):
        for n in (512, 700, 1000, 4096, 16384):
            assert native.gmt_connection_radius(n, d, 0.0, 1.0) == O.radius_thm1(n, d, 0.0, 1.0)


def test_invalid_arguments_are_rejected_without_gpu(native):
    import ctypes as C
    sp = native.gmt_space()
    sp.kind, sp.dim, sp.pos_dim = 0, 11, 11
    b = native.gmt_boxes()
    g = native.gmt_goal()
    p = native.gmt_params()
    h = C.c_void_p(None)
    xi = (C.c_float * 10)()
    st = native.lib.gmt_build_graph(C.byref(sp), C.byref(b), C.cast(xi, C.c_void_p), C.byref(g), C.byref(p),
                                    C.byref(h), None)
    assert st == native.GMT_ERR_INVALID and "dim" in native.gmt_last_error()
    sp.dim = sp.pos_dim = 2
    sp.lo[0] = sp.lo[1] = 0.0
    sp.hi[0] = sp.hi[1] = 1.0
    p.n, p.r, p.lambda_ = 10, 0.1, 1.5
    st = native.lib.gmt_build_graph(C.byref(sp), C.byref(b), C.cast(xi, C.c_void_p), C.byref(g), C.byref(p),
                                    C.byref(h), None)
    assert st == native.GMT_ERR_INVALID and "lambda" in native.gmt_last_error()
    assert native.lib.gmt_plan(None, C.byref(b), C.byref(p), None, None, None, None, None) == native.GMT_ERR_INVALID
