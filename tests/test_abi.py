"""The C ABI library builds, loads and exports every entry point include/psc.h declares.

No GPU needed: only calls that fail on argument checks before touching CUDA run here.
"""
import os
import re

import pytest

import paper_1605_03726_gb300 as psc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    with open(os.path.join(ROOT, "include", "psc.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(psc_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported():
    names = declared()
    assert "psc_run" in names and "psc_populate" in names
    L = psc.lib()
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(psc.EXPORTED) | set(names)


def test_host_side_argument_checks():
    import ctypes
    L = psc.lib()
    h = ctypes.c_void_p()
    assert L.psc_lattice_create(ctypes.byref(h), 8, 5, 8, 1e-8, 7, 0, None) == psc.E_DIMS
    assert L.psc_lattice_create(ctypes.byref(h), 8, 8, 7, 1e-8, 7, 0, None) == psc.E_DIMS
    assert L.psc_lattice_create(ctypes.byref(h), 2, 8, 8, 1e-8, 7, 0, None) == psc.E_DIMS
    assert L.psc_lattice_create(ctypes.byref(h), 2048, 1024, 1024, 1e-8, 7, 0, None) == psc.E_DIMS
    assert L.psc_lattice_create(ctypes.byref(h), 8, 8, 8, -1.0, 7, 0, None) == psc.E_ARG
    assert L.psc_lattice_create(None, 8, 8, 8, 1e-8, 7, 0, None) == psc.E_ARG
    assert L.psc_run(None, 1.0) == psc.E_ARG
    assert L.psc_status_string(psc.E_CAPACITY) == b"PSC_E_CAPACITY"


def test_library_is_built_for_sm_103a():
    from paper_1605_03726_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH
    assert os.path.exists(build.LIB)
