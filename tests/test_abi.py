"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/thm.h declares; argument errors come back as codes, not crashes.
No compute call is made here (no GPU on this side)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2105_11993_gb300 import build as B
    B.build()
    import paper_2105_11993_gb300 as thm
    return thm.load()


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "thm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(thm_[a-z_]+)\s*\(", txt)))


def test_header_and_binding_agree():
    import paper_2105_11993_gb300 as thm
    assert header_symbols() == sorted(thm.symbols)


def test_library_exports_every_declared_symbol(lib):
    for name in header_symbols():
        assert hasattr(lib, name), name


def test_invalid_arguments_return_codes(lib):
    h = C.c_void_p()
    coords = np.zeros((4, 2))
    cells = np.zeros((1, 4), np.int64)
    sub = np.zeros(1, np.int32)
    rc = lib.thm_mesh_create(C.byref(h), 4, 1, 4, coords.ctypes.data_as(C.c_void_p), 1,
                             cells.ctypes.data_as(C.c_void_p), sub.ctypes.data_as(C.c_void_p), 0, None, None, 0)
    assert rc == -1 and b"dim" in lib.thm_last_error()
    rc = lib.thm_mesh_create(C.byref(h), 3, 2, 4, coords.ctypes.data_as(C.c_void_p), 1,
                             cells.ctypes.data_as(C.c_void_p), sub.ctypes.data_as(C.c_void_p), 0, None, None, 0)
    assert rc == -1 and b"order" in lib.thm_last_error()
    rc = lib.thm_ddm_solve(None, None, None, None)
    assert rc == -1


def test_no_gpu_is_an_error_not_a_fallback(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import workloads as W
    m = W.structured_mesh_2d(2, 2)
    h = C.c_void_p()
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    rc = lib.thm_mesh_create(C.byref(h), 2, 1, m.n_vert, p(m.coords), m.n_cell, p(m.cells),
                             p(m.cell_sub), m.bfaces.shape[0], p(m.bfaces), p(m.btag), 0)
    assert rc == -6 and b"CUDA" in lib.thm_last_error()
