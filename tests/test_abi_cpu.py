"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/ibm.h declares; host-side validation runs without a GPU."""
import ctypes
import os
import re

import pytest

from paper_1612_03399_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ibm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ibm_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    syms = declared_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(lib, s), s
    # and the binding knows the signature of each
    assert set(syms) == set(_lib.SIGNATURES)


def test_create_without_gpu_fails_loudly():
    """No CUDA device here: creation must fail with a CUDA status, never fall
    back to a CPU path."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = _lib.library()
    h = ctypes.c_void_p()
    st = lib.ibm_create_bodies(ctypes.byref(h), None, 0, None, None, 0)
    assert st == 1                               # null arguments are rejected first
    assert lib.ibm_last_error(None)
    from paper_1612_03399_gb300 import workloads as W
    wl = W.single_drop(level=1, n=16)
    with pytest.raises(RuntimeError):
        _lib.Context(wl.bodies, wl.grid)


def test_flow_create_validates_before_touching_the_device():
    """Grid and parameter checks of ibm_flow_create come before any CUDA call:
    a grid of 2^31 cells or more (the stencils' 32-bit neighbour offsets) is
    refused as unsupported, a grid below four cells per direction as invalid."""
    lib = _lib.library()
    h = ctypes.c_void_p()
    g = _lib.GridDesc()
    for k, n in enumerate((2048, 2048, 512)):
        g.n[k] = n
        g.L[k] = 1.0
    assert lib.ibm_flow_create(ctypes.byref(g), 0.1, 1e-3, ctypes.byref(h)) == 6
    assert b"2^31" in lib.ibm_last_error(None)
    g.n[2] = 3
    assert lib.ibm_flow_create(ctypes.byref(g), 0.1, 1e-3, ctypes.byref(h)) == 1
    assert not h.value
