"""The C-ABI library builds, loads and exports every entry point of include/gridpf.h (no GPU needed)."""
import ctypes

import pytest

from paper_2102_11910_gb300 import _native, build


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    L = ctypes.CDLL(path)
    declared = _native.declared_functions()
    assert "pf_plan_create" in declared and "pf_vic_velocity" in declared
    for name in declared:
        assert hasattr(L, name), name
    # the binding knows the signature of every declared function and nothing else
    assert sorted(_native.SIGNATURES) == declared


def test_null_arguments_are_rejected_without_touching_the_gpu():
    L = _native.lib()
    assert L.pf_plan_create(None, None, None) == 1          # PF_ERR_ARG
    assert L.pf_sync(None, None) == 1
    assert L.pf_regularize(None, None, None, None, 0, None) == 1
    assert L.pf_vic_velocity_host(None, None, None, None, 1, 0.0, 0.0, None, None) == 1
    assert L.pf_vic_velocity_host_async(None, None, None, None, 1, 0.0, 0.0, None, None) == 1
    desc = _native.PfGridDesc(4, 4, 0.1, 0.0, 0.0, 0)      # nx < 8
    h = ctypes.c_void_p()
    assert L.pf_plan_create(ctypes.byref(desc), None, ctypes.byref(h)) == 1
    desc = _native.PfGridDesc(64, 64, -1.0, 0.0, 0.0, 0)   # dx <= 0
    assert L.pf_plan_create(ctypes.byref(desc), None, ctypes.byref(h)) == 1
    desc = _native.PfGridDesc(64, 64, 0.1, 0.0, 0.0, 7)    # bad precision
    assert L.pf_plan_create(ctypes.byref(desc), None, ctypes.byref(h)) == 1


def test_header_is_plain_c_and_cpp():
    """include/gridpf.h compiles as C99 and as C++ with warnings as errors:
    the boundary carries no C++ or torch types."""
    import os
    import shutil
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    hdr = os.path.join(root, "include", "gridpf.h")
    for cc, lang, std in (("gcc", "c", "-std=c99"), ("g++", "c++", "-std=c++17")):
        if shutil.which(cc) is None:
            pytest.skip("%s not installed" % cc)
        r = subprocess.run([cc, "-fsyntax-only", std, "-Wall", "-Wextra", "-Werror", "-x", lang, hdr],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
