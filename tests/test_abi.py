"""The C-ABI library builds, loads and exports every function that
include/hyb.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_1509_01399_gb300", "libhyb.so")


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(hyb_\w+)\s*\(", txt, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_1509_01399_gb300 import build
        build.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hyb_mesh_create", "hyb_forward", "hyb_adjoint", "hyb_gradient", "hyb_cg_step"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (hyb_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_binding_mirrors_the_abi(lib):
    from paper_1509_01399_gb300 import hyb
    for n in declared_functions():
        assert n in hyb.EXPORTED and callable(getattr(hyb, n))
    assert hyb.hyb_last_error() == ""


def test_binding_structs_match_the_c_layout(tmp_path):
    """Every struct of the binding has the size and field offsets the C
    compiler gives the declarations of include/hyb.h."""
    from paper_1509_01399_gb300 import hyb
    structs = [hyb.hyb_mesh_desc, hyb.hyb_mesh_info, hyb.hyb_source, hyb.hyb_cg_params, hyb.hyb_cg_state,
               hyb.hyb_cg_report]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hyb.h"', "int main(void) {"]
    for st in structs:
        n = st.__name__
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (n, n))
        for f, _ in st._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (n, f, n, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(ln.split() for ln in subprocess.run([str(exe)], capture_output=True, text=True,
                                                   check=True).stdout.splitlines())
    for st in structs:
        n = st.__name__
        assert int(out[n]) == ctypes.sizeof(st), n
        for f, _ in st._fields_:
            assert int(out[n + "." + f]) == getattr(st, f).offset, (n, f)


def test_argument_errors_need_no_gpu(lib):
    from paper_1509_01399_gb300 import hyb
    d = hyb.hyb_mesh_desc()
    d.n[0] = 2  # invalid: every axis needs 3 nodes
    with pytest.raises(hyb.HybError) as e:
        hyb.hyb_mesh_create(d, 0)
    assert e.value.status == hyb.HYB_ERR_ARG
    assert "n[0]" in hyb.hyb_last_error()
