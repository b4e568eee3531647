"""CPU checks of the C ABI: the library loads, exports every entry point include/sccs.h
declares, and rejects bad inputs before it touches a GPU."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sccs.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__._build_module().build()
    import paper_1208_0945_gb300 as P
    return P


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sccs_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sccs_create", "sccs_destroy", "sccs_set_prior", "sccs_fit", "sccs_grad_hess",
                     "sccs_last_error", "sccs_logpost"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    import ctypes
    so = ctypes.CDLL(os.path.join(ROOT, "paper_1208_0945_gb300", "_lib", "libsccs.so"))
    for name in declared_functions():
        assert hasattr(so, name), name
    assert set(declared_functions()) == set(lib.EXPORTED)


def test_version(lib):
    v, s = lib.sccs_version()
    assert v == 1 and "sm_103a" in s


def _tiny():
    pid = np.array([0, 0, 1, 1, 2], np.int64)
    y = np.array([1, 0, 0, 2, 1], np.int32)
    L = np.array([10.0, 20.0, 5.0, 5.0, 7.0])
    col_ptr = np.array([0, 2, 3], np.int64)
    rows = np.array([0, 3, 4], np.int32)
    return pid, y, L, col_ptr, rows


@pytest.mark.parametrize("mutate,code", [
    ("unsorted", -2), ("neg_y", -1), ("zero_L", -1), ("nan_L", -1), ("row_oob", -1),
    ("col_ptr_decreasing", -1), ("col_ptr_start", -1), ("nonbinary", -3), ("no_events", -1),
])
def test_validation_errors_need_no_gpu(lib, mutate, code):
    pid, y, L, cp, rows = _tiny()
    xv = None
    if mutate == "unsorted":
        pid = pid[::-1].copy()
    elif mutate == "neg_y":
        y[1] = -1
    elif mutate == "zero_L":
        L[2] = 0.0
    elif mutate == "nan_L":
        L[2] = np.nan
    elif mutate == "row_oob":
        rows[1] = 5
    elif mutate == "col_ptr_decreasing":
        cp = np.array([0, 3, 2], np.int64)
    elif mutate == "col_ptr_start":
        cp = np.array([1, 2, 3], np.int64)
    elif mutate == "nonbinary":
        xv = np.array([1.0, 2.0, 1.0])
    elif mutate == "no_events":
        y[:] = 0
    with pytest.raises(lib.SCCSError) as ei:
        lib.sccs_create(5, pid, y, L, 2, cp, rows, xv)
    assert ei.value.code == code
    assert lib.sccs_last_error(None)


@pytest.mark.parametrize("field,value", [("max_inflight", 0), ("queue_capacity", 0), ("hbm_budget_bytes", -1),
                                         ("struct_size", 8)])
def test_server_options_rejected_before_cuda(lib, field, value):
    import ctypes
    from paper_1208_0945_gb300 import sccs as S
    o = S.sccs_server_opts(struct_size=ctypes.sizeof(S.sccs_server_opts), device=0, max_inflight=4,
                           queue_capacity=4, hbm_budget_bytes=0)
    setattr(o, field, value)
    srv = ctypes.c_void_p()
    assert S._lib.sccs_server_create(ctypes.byref(srv), ctypes.byref(o)) == -1
    assert srv.value is None
    assert S._lib.sccs_submit(None, None, None) == -1
    assert S._lib.sccs_server_destroy(None) == 0
