"""The C-ABI library builds, loads and exports every function that
include/lpsim.h declares; argument checks that need no GPU."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        with open(os.path.join(ROOT, "include", fn)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(lpsim_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import paper_2406_08496_gb300 as L
    L.build()
    return L.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 18
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    import paper_2406_08496_gb300 as L
    assert sorted(L.EXPORTED) == names


def test_version_and_empty_error(lib):
    assert b"sm_103a" in lib.lpsim_version()
    assert isinstance(lib.lpsim_last_error(), bytes)


def test_argument_checks_without_gpu(lib):
    import paper_2406_08496_gb300 as L
    P = ctypes.c_void_p
    # one allocator callback without the other
    assert lib.lpsim_set_allocator(L.ALLOC_T(lambda s, u: None), ctypes.cast(None, L.FREE_T), None) == -1
    # no output handle
    p = L.Params(**L.DEFAULT_PARAMS)
    assert lib.lpsim_load_network(None, None, ctypes.byref(p), None) == -1
    # 5 lanes is rejected before any device work
    src = np.array([0], np.uint32)
    dst = np.array([1], np.uint32)
    ln = np.array([100.0], np.float32)
    lanes = np.array([5], np.uint8)
    vmax = np.array([10.0], np.float32)
    green = np.zeros(2, np.uint32)
    net = L.Network(2, 1, *(P(a.ctypes.data) for a in (src, dst, ln, lanes, vmax, green)), None)
    h = P()
    assert lib.lpsim_load_network(ctypes.byref(h), ctypes.byref(net), ctypes.byref(p), None) == -1
    assert b"lanes" in lib.lpsim_last_error()
    # bad model parameter
    bad = L.Params(**dict(L.DEFAULT_PARAMS, dt=0.0))
    lanes[0] = 2
    assert lib.lpsim_load_network(ctypes.byref(h), ctypes.byref(net), ctypes.byref(bad), None) == -1
    # the allocation-free query refuses more vehicles than its fixed scratch
    lib.lpsim_get_state_noalloc.argtypes = [P, ctypes.c_uint64, P, P, P, P, P, P]
    assert lib.lpsim_get_state_noalloc(None, 1048577, None, None, None, None, None, None) == -1
    assert b"exceed" in lib.lpsim_last_error()


def test_binding_refuses_without_library(tmp_path):
    import paper_2406_08496_gb300 as L
    saved = L._lib
    try:
        L._lib = None
        with pytest.raises(ImportError):
            L.load_library(str(tmp_path / "missing.so"))
    finally:
        L._lib = saved
