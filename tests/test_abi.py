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
    # struct sizes agree with the C layout (natural alignment)
    assert ctypes.sizeof(hyb.hyb_source) == 24
    assert ctypes.sizeof(hyb.hyb_mesh_desc) == 4 * 3 + 4 + 8 + 24 + 12 + 12 + 24 + 4 + 4 + 8 + 8
    assert hyb.hyb_last_error() == ""


def test_argument_errors_need_no_gpu(lib):
    from paper_1509_01399_gb300 import hyb
    d = hyb.hyb_mesh_desc()
    d.n[0] = 2  # invalid: every axis needs 3 nodes
    with pytest.raises(hyb.HybError) as e:
        hyb.hyb_mesh_create(d, 0)
    assert e.value.status == hyb.HYB_ERR_ARG
    assert "n[0]" in hyb.hyb_last_error()
