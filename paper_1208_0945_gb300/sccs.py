"""ctypes binding of libsccs.so: the C ABI of include/sccs.h, one Python name per entry point.

Only argument marshalling happens here; every step of the fit runs in the library's CUDA
kernels.  There is no CPU fallback: if the library is missing this module raises at import.
PyTorch, when present, only supplies the CUDA stream (and optionally the allocator).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libsccs.so")

OK, NOT_CONVERGED, PENDING = 0, 1, 2
E_INVAL, E_UNSORTED, E_NONBINARY, E_NOMEM, E_CUDA = -1, -2, -3, -4, -5
E_TIMEOUT, E_NUMERIC, E_BUSY, E_DUPLICATE, E_UNSUPPORTED = -6, -7, -8, -9, -10
PRIOR = {"none": 0, "normal": 1, "laplace": 2}
TOL = {"abs_logpost": 0, "rel_logpost": 1, "genkin_xbeta": 2}
PREC = {"fp64": 0, "fp32_polish": 1, "fp32": 2}

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
_lib = ctypes.CDLL(LIB_PATH)

_alloc_fn = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_free_fn = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class sccs_create_opts(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_int32), ("device", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("num_shards", ctypes.c_int32), ("threads_per_block", ctypes.c_int32),
                ("alloc", _alloc_fn), ("free", _free_fn), ("alloc_ctx", ctypes.c_void_p),
                ("narrow_max_nnz", ctypes.c_int32), ("narrow_group_max", ctypes.c_int32),
                ("cluster_ctas", ctypes.c_int32), ("cluster_max_nnz", ctypes.c_int32)]


class sccs_data_info(ctypes.Structure):
    _fields_ = [("rows_in", ctypes.c_int64), ("rows_kept", ctypes.c_int64), ("subjects_in", ctypes.c_int64),
                ("subjects_kept", ctypes.c_int64), ("nnz_kept", ctypes.c_int64), ("segments", ctypes.c_int64),
                ("max_column_nnz", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("upload_bytes", ctypes.c_int64),
                ("columns", ctypes.c_int32), ("num_shards", ctypes.c_int32),
                ("threads_per_block", ctypes.c_int32), ("narrow_columns", ctypes.c_int32),
                ("cluster_ctas", ctypes.c_int32), ("cluster_columns", ctypes.c_int32)]


class sccs_fit_opts(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_int32), ("warm_start", ctypes.c_int32),
                ("beta0", ctypes.POINTER(ctypes.c_double)), ("tol_mode", ctypes.c_int32),
                ("max_cycles", ctypes.c_int32), ("tol", ctypes.c_double), ("precision", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("logpost_history", ctypes.POINTER(ctypes.c_double)),
                ("subject_weights", ctypes.POINTER(ctypes.c_int32))]


class sccs_fit_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("cycles", ctypes.c_int32), ("steps", ctypes.c_int64),
                ("nonzero_steps", ctypes.c_int64), ("logpost", ctypes.c_double), ("conv_value", ctypes.c_double),
                ("kernel_ms", ctypes.c_double), ("total_ms", ctypes.c_double), ("warnings", ctypes.c_int32),
                ("fp32_cycles", ctypes.c_int32)]


class sccs_server_opts(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_int32), ("device", ctypes.c_int32), ("max_inflight", ctypes.c_int32),
                ("queue_capacity", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_int64)]


class sccs_request(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_int32), ("prior_type", ctypes.c_int32), ("dataset", ctypes.c_void_p),
                ("variance", ctypes.c_double), ("tol_mode", ctypes.c_int32), ("max_cycles", ctypes.c_int32),
                ("tol", ctypes.c_double), ("precision", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("beta0", ctypes.POINTER(ctypes.c_double)), ("subject_weights", ctypes.POINTER(ctypes.c_int32)),
                ("heldout_weights", ctypes.POINTER(ctypes.c_int32)), ("dataset_alt", ctypes.c_void_p)]


class sccs_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("cycles", ctypes.c_int32), ("fp32_cycles", ctypes.c_int32),
                ("team", ctypes.c_int32), ("logpost", ctypes.c_double), ("queue_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double), ("beta", ctypes.POINTER(ctypes.c_double)),
                ("heldout_loglik", ctypes.c_double)]


class sccs_server_stats(ctypes.Structure):
    _fields_ = [("pending", ctypes.c_int64), ("running", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("slot_bytes", ctypes.c_int64), ("ctas_in_use", ctypes.c_int32), ("capacity_ctas", ctypes.c_int32)]


_P = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_SIGS = {
    "sccs_version": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_char_p)]),
    "sccs_last_error": (ctypes.c_char_p, [_P]),
    "sccs_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int64, _P, _P, _P, ctypes.c_int32, _P, _P, _P,
                                   ctypes.POINTER(sccs_create_opts)]),
    "sccs_destroy": (ctypes.c_int, [_P]),
    "sccs_get_info": (ctypes.c_int, [_P, ctypes.POINTER(sccs_data_info)]),
    "sccs_set_prior": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_double]),
    "sccs_fit": (ctypes.c_int, [_P, ctypes.POINTER(sccs_fit_opts), _dp, ctypes.POINTER(sccs_fit_info)]),
    "sccs_grad_hess": (ctypes.c_int, [_P, ctypes.c_int32, _dp, _dp, _dp]),
    "sccs_fit_batch": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32, ctypes.POINTER(sccs_fit_opts),
                                      ctypes.POINTER(_dp), ctypes.POINTER(sccs_fit_info)]),
    "sccs_logpost": (ctypes.c_int, [_P, _dp, _dp, _dp]),
    "sccs_get_beta": (ctypes.c_int, [_P, _dp]),
    "sccs_heldout_loglik": (ctypes.c_int, [_P, _dp, _P, _dp]),
    "sccs_selftest_exp": (ctypes.c_int, [ctypes.c_int32, _dp, ctypes.c_int64, _dp, _dp]),
    "sccs_selftest_div": (ctypes.c_int, [ctypes.c_int32, _dp, _dp, ctypes.c_int64, _dp, _dp]),
    "sccs_check_wait_timeout": (ctypes.c_int, [_P, ctypes.c_double]),
    "sccs_debug_layout": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "sccs_grad_hess_noalloc": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, ctypes.c_double, ctypes.c_int64, _P, _P]),
    "sccs_server_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(sccs_server_opts)]),
    "sccs_submit": (ctypes.c_int, [_P, ctypes.POINTER(sccs_request), ctypes.POINTER(ctypes.c_uint64)]),
    "sccs_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(sccs_result)]),
    "sccs_server_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(sccs_server_stats)]),
    "sccs_server_destroy": (ctypes.c_int, [_P]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


class SCCSError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = sccs_last_error(None)
        super().__init__(f"{where} returned {code}: {msg}")
        self.code = code


def _check(code: int, where: str) -> int:
    if code < 0:
        raise SCCSError(code, where)
    return code


def _ptr(a: np.ndarray | None):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _dptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(_dp)


def _weights(w):
    """Subject weights (one non-negative integer per input subject) as an int32 array, or None."""
    return None if w is None else np.ascontiguousarray(w, np.int32)


def _iptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


# ------------------------------------------------------------------ the C ABI, name for name

def sccs_version() -> tuple[int, str]:
    v = ctypes.c_int32()
    s = ctypes.c_char_p()
    _lib.sccs_version(ctypes.byref(v), ctypes.byref(s))
    return v.value, s.value.decode()


def sccs_last_error(handle) -> str:
    r = _lib.sccs_last_error(handle)
    return r.decode() if r else ""


def sccs_create(K, patient_id, y, offset_L, J, col_ptr, row_idx, x_values=None, *, device=0, stream=None,
                num_shards=0, threads_per_block=0, narrow_max_nnz=0, narrow_group_max=0, cluster_ctas=0,
                cluster_max_nnz=0):
    """Returns an opaque handle (int).  Arrays are copied by the library before it returns."""
    pid = np.ascontiguousarray(patient_id, np.int64)
    yy = np.ascontiguousarray(y, np.int32)
    LL = np.ascontiguousarray(offset_L, np.float64)
    cp = np.ascontiguousarray(col_ptr, np.int64)
    ri = np.ascontiguousarray(row_idx, np.int32)
    xv = None if x_values is None else np.ascontiguousarray(x_values, np.float64)
    o = sccs_create_opts(struct_size=ctypes.sizeof(sccs_create_opts), device=int(device),
                         stream=stream, num_shards=int(num_shards), threads_per_block=int(threads_per_block),
                         narrow_max_nnz=int(narrow_max_nnz), narrow_group_max=int(narrow_group_max),
                         cluster_ctas=int(cluster_ctas), cluster_max_nnz=int(cluster_max_nnz))
    h = ctypes.c_void_p()
    _check(_lib.sccs_create(ctypes.byref(h), int(K), _ptr(pid), _ptr(yy), _ptr(LL), int(J), _ptr(cp), _ptr(ri),
                            _ptr(xv), ctypes.byref(o)), "sccs_create")
    return h.value


def sccs_destroy(handle) -> int:
    return _lib.sccs_destroy(handle)


def sccs_get_info(handle) -> dict:
    info = sccs_data_info()
    _check(_lib.sccs_get_info(handle, ctypes.byref(info)), "sccs_get_info")
    return {name: getattr(info, name) for name, _ in sccs_data_info._fields_ if name != "reserved"}


def sccs_set_prior(handle, prior: str | int, variance: float = 1.0) -> int:
    pt = PRIOR[prior] if isinstance(prior, str) else int(prior)
    return _check(_lib.sccs_set_prior(handle, pt, float(variance)), "sccs_set_prior")


def sccs_fit(handle, J: int, *, beta0=None, warm_start=False, tol_mode="rel_logpost", tol=1e-12,
             max_cycles=1000, precision="fp64", history=False, weights=None) -> dict:
    b0 = None if beta0 is None else np.ascontiguousarray(beta0, np.float64)
    hist = np.full(max_cycles + 1, np.nan) if history else None
    w = _weights(weights)
    o = sccs_fit_opts(struct_size=ctypes.sizeof(sccs_fit_opts), warm_start=int(bool(warm_start)),
                      beta0=_dptr(b0), tol_mode=TOL[tol_mode], max_cycles=int(max_cycles), tol=float(tol),
                      precision=PREC[precision], logpost_history=_dptr(hist), subject_weights=_iptr(w))
    beta = np.zeros(max(J, 1))
    info = sccs_fit_info()
    rc = _check(_lib.sccs_fit(handle, ctypes.byref(o), _dptr(beta), ctypes.byref(info)), "sccs_fit")
    out = {name: getattr(info, name) for name, _ in sccs_fit_info._fields_ if name != "reserved"}
    out["rc"] = rc
    out["beta"] = beta[:J]
    if history:
        out["history"] = hist[:info.cycles + 1]
    return out


def sccs_fit_batch(handles, Js, *, warm_start=False, tol_mode="rel_logpost", tol=1e-12, max_cycles=1000,
                   precision="fp64") -> list:
    """One persistent launch for several fits (one per handle); returns one result dict per fit."""
    n = len(handles)
    o = sccs_fit_opts(struct_size=ctypes.sizeof(sccs_fit_opts), warm_start=int(bool(warm_start)), beta0=None,
                      tol_mode=TOL[tol_mode], max_cycles=int(max_cycles), tol=float(tol), precision=PREC[precision],
                      logpost_history=None)
    hs = (_P * n)(*handles)
    betas = [np.zeros(max(J, 1)) for J in Js]
    bptr = (_dp * n)(*[b.ctypes.data_as(_dp) for b in betas])
    infos = (sccs_fit_info * n)()
    rc = _lib.sccs_fit_batch(hs, n, ctypes.byref(o), bptr, infos)
    out = []
    for k in range(n):
        d = {name: getattr(infos[k], name) for name, _ in sccs_fit_info._fields_}
        d["beta"] = betas[k][:Js[k]]
        out.append(d)
    _check(rc, "sccs_fit_batch")
    return out


def sccs_grad_hess(handle, j: int, beta=None) -> tuple[float, float]:
    b = None if beta is None else np.ascontiguousarray(beta, np.float64)
    g, h = ctypes.c_double(), ctypes.c_double()
    _check(_lib.sccs_grad_hess(handle, int(j), _dptr(b), ctypes.byref(g), ctypes.byref(h)), "sccs_grad_hess")
    return g.value, h.value


def sccs_logpost(handle, beta=None) -> tuple[float, float]:
    b = None if beta is None else np.ascontiguousarray(beta, np.float64)
    lp, ll = ctypes.c_double(), ctypes.c_double()
    _check(_lib.sccs_logpost(handle, _dptr(b), ctypes.byref(lp), ctypes.byref(ll)), "sccs_logpost")
    return lp.value, ll.value


def sccs_heldout_loglik(handle, weights=None, beta=None) -> float:
    """Eq. 2 with subject i counted weights[i] times (a held-out fold's mask) at beta, or at the
    handle's current beta (after a fit: its MAP) when beta is None."""
    b = None if beta is None else np.ascontiguousarray(beta, np.float64)
    w = _weights(weights)
    ll = ctypes.c_double()
    _check(_lib.sccs_heldout_loglik(handle, _dptr(b), None if w is None else ctypes.c_void_p(w.ctypes.data),
                                    ctypes.byref(ll)), "sccs_heldout_loglik")
    return ll.value


def sccs_selftest_exp(x, device=0):
    """(the library's e^x used in the coordinate step, CUDA's exp) on the values x."""
    xx = np.ascontiguousarray(x, np.float64)
    ours, ref = np.empty_like(xx), np.empty_like(xx)
    _check(_lib.sccs_selftest_exp(int(device), _dptr(xx), xx.size, _dptr(ours), _dptr(ref)), "sccs_selftest_exp")
    return ours, ref


def sccs_selftest_div(a, b, device=0):
    """(the library's quotient a/b used in the coordinate step, CUDA's IEEE division)."""
    aa = np.ascontiguousarray(a, np.float64)
    bb = np.ascontiguousarray(b, np.float64)
    if aa.shape != bb.shape:
        raise ValueError("a and b must have the same shape")
    ours, ref = np.empty_like(aa), np.empty_like(aa)
    _check(_lib.sccs_selftest_div(int(device), _dptr(aa), _dptr(bb), aa.size, _dptr(ours), _dptr(ref)),
           "sccs_selftest_div")
    return ours, ref


def sccs_get_beta(handle, J: int) -> np.ndarray:
    b = np.zeros(max(J, 1))
    _check(_lib.sccs_get_beta(handle, _dptr(b)), "sccs_get_beta")
    return b[:J]


def sccs_check_wait_timeout(handle, timeout_ms: float) -> int:
    """Returns the raw status; E_TIMEOUT (-6) is the expected result."""
    return _lib.sccs_check_wait_timeout(handle, float(timeout_ms))


DBG = {name: i + 1 for i, name in enumerate(
    "PAT_PTR NEV L YTX ROWS SEGS GRP_BASE SLICE_ROW SLICE_SEG SLICE_GRP SHARD_ROW SHARD_PAT YCOL_PTR YSUB YCNT "
    "NARROW NEXT_WIDE NAR_PTR NAR_SEG NAR_ROW NAR_GROUP CCLS NEXT_GRID CGROUP CROWS CSEGS CGRP_BASE CSLICE_ROW "
    "CSLICE_SEG CSLICE_GRP CSHARD_ROW CSHARD_PAT KEPT_FROM ROW_PTR ROW_COL SCALARS".split())}
_DBG_TYPES = {"NEV": np.int32, "ROWS": np.int32, "YSUB": np.int32, "YCNT": np.int32, "NEXT_WIDE": np.int32,
              "NAR_ROW": np.int32, "NAR_GROUP": np.int32, "NEXT_GRID": np.int32, "CGROUP": np.int32,
              "CROWS": np.int32, "ROW_COL": np.int32, "SEGS": np.int32, "CSEGS": np.int32, "NAR_SEG": np.int32,
              "NARROW": np.uint8, "CCLS": np.uint8, "L": np.float64, "YTX": np.float64}


def sccs_debug_layout(handle, name: str) -> np.ndarray:
    """One array of the handle's layout (a test diagnostic); SEGS / CSEGS come back as (n, 2) and
    NAR_SEG as (n, 4) int32."""
    which = DBG[name]
    nbytes = ctypes.c_int64()
    _check(_lib.sccs_debug_layout(handle, which, None, 0, ctypes.byref(nbytes)), "sccs_debug_layout")
    dt = _DBG_TYPES.get(name, np.int64)
    out = np.empty(nbytes.value // np.dtype(dt).itemsize, dt)
    if out.size:
        _check(_lib.sccs_debug_layout(handle, which, out.ctypes.data, nbytes.value, ctypes.byref(nbytes)),
               "sccs_debug_layout")
    if name in ("SEGS", "CSEGS"):
        return out.reshape(-1, 2)
    if name == "NAR_SEG":
        return out.reshape(-1, 4)
    return out


NOALLOC_MAX_SEGMENTS = 1048576


def sccs_grad_hess_noalloc(seg_ptr, seg_subject, rows, E, D, n, ytx: float, P: int, gh_out, stream=None) -> int:
    """g_j, h_j of one column from device arrays the caller holds, allocating nothing on the
    device (for callers that cannot allocate at that point).  Pointer arguments are device
    addresses (ints); writes g_j, h_j to gh_out[0:2].  Asynchronous on `stream`; returns the
    status (0 on success) and raises on errors."""
    return _check(_lib.sccs_grad_hess_noalloc(seg_ptr, seg_subject, rows, E, D, n, float(ytx), int(P), gh_out,
                                              stream), "sccs_grad_hess_noalloc")


def sccs_server_create(device=0, max_inflight=64, queue_capacity=4096, hbm_budget_bytes=0):
    o = sccs_server_opts(struct_size=ctypes.sizeof(sccs_server_opts), device=int(device),
                         max_inflight=int(max_inflight), queue_capacity=int(queue_capacity),
                         hbm_budget_bytes=int(hbm_budget_bytes))
    srv = ctypes.c_void_p()
    _check(_lib.sccs_server_create(ctypes.byref(srv), ctypes.byref(o)), "sccs_server_create")
    return srv.value


def sccs_submit(server, dataset, prior="normal", variance=1.0, tol_mode="rel_logpost", tol=1e-12,
                max_cycles=1000, precision="fp64", beta0=None, weights=None, heldout_weights=None,
                dataset_alt=None) -> int:
    b0 = None if beta0 is None else np.ascontiguousarray(beta0, np.float64)
    w, wh = _weights(weights), _weights(heldout_weights)
    r = sccs_request(struct_size=ctypes.sizeof(sccs_request), prior_type=PRIOR[prior], dataset=dataset,
                     variance=float(variance), tol_mode=TOL[tol_mode], max_cycles=int(max_cycles), tol=float(tol),
                     precision=PREC[precision], reserved=0, beta0=_dptr(b0), subject_weights=_iptr(w),
                     heldout_weights=_iptr(wh), dataset_alt=dataset_alt)
    t = ctypes.c_uint64()
    _check(_lib.sccs_submit(server, ctypes.byref(r), ctypes.byref(t)), "sccs_submit")
    return t.value


def sccs_poll(server, ticket: int, J: int):
    """None while pending; else the result dict (beta included)."""
    beta = np.zeros(max(J, 1))
    res = sccs_result(beta=_dptr(beta))
    rc = _check(_lib.sccs_poll(server, ctypes.c_uint64(ticket), ctypes.byref(res)), "sccs_poll")
    if rc == PENDING:
        return None
    out = {name: getattr(res, name) for name, _ in sccs_result._fields_ if name not in ("reserved", "beta")}
    out["beta"] = beta[:J]
    return out


def sccs_server_get_stats(server) -> dict:
    st = sccs_server_stats()
    _check(_lib.sccs_server_get_stats(server, ctypes.byref(st)), "sccs_server_get_stats")
    return {name: getattr(st, name) for name, _ in sccs_server_stats._fields_}


def sccs_server_destroy(server) -> int:
    return _lib.sccs_server_destroy(server)


class FitServer:
    """Continuous-batching fit server over resident datasets (SCCSModel handles)."""

    def __init__(self, device=0, max_inflight=64, queue_capacity=4096, hbm_budget_bytes=0):
        self.server = sccs_server_create(device, max_inflight, queue_capacity, hbm_budget_bytes)
        self._J = {}

    def submit(self, model, alt=None, **kw) -> int:
        """alt: another SCCSModel of the same data with a different shard count (see dataset_alt)."""
        t = sccs_submit(self.server, model.handle, dataset_alt=None if alt is None else alt.handle, **kw)
        self._J[t] = model.J
        return t

    def poll(self, ticket):
        r = sccs_poll(self.server, ticket, self._J[ticket])
        if r is not None:
            del self._J[ticket]
        return r

    def wait(self, ticket, timeout_s=120.0):
        import time
        t0 = time.perf_counter()
        while True:
            r = self.poll(ticket)
            if r is not None:
                return r
            if time.perf_counter() - t0 > timeout_s:
                raise TimeoutError(f"request {ticket} still pending after {timeout_s} s")
            time.sleep(0.0002)

    def stats(self) -> dict:
        return sccs_server_get_stats(self.server)

    def close(self):
        if getattr(self, "server", None):
            sccs_server_destroy(self.server)
            self.server = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ convenience wrapper

def _torch_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return None


class SCCSModel:
    """One dataset resident on the GPU, fitted through the C ABI."""

    def __init__(self, data=None, *, K=None, patient_id=None, y=None, L=None, J=None, col_ptr=None,
                 row_idx=None, x_values=None, device=0, stream="torch", num_shards=0, threads_per_block=0,
                 narrow_max_nnz=0, narrow_group_max=0, cluster_ctas=0, cluster_max_nnz=0):
        if data is not None:
            K, patient_id, y, L, J = data.K, data.patient_id, data.y, data.L, data.J
            col_ptr, row_idx = data.col_ptr, data.row_idx
        st = _torch_stream() if stream == "torch" else stream
        self.J = int(J)
        self.device = int(device)
        self.handle = sccs_create(K, patient_id, y, L, J, col_ptr, row_idx, x_values, device=device, stream=st,
                                  num_shards=num_shards, threads_per_block=threads_per_block,
                                  narrow_max_nnz=narrow_max_nnz, narrow_group_max=narrow_group_max,
                                  cluster_ctas=cluster_ctas, cluster_max_nnz=cluster_max_nnz)

    def close(self):
        if getattr(self, "handle", None):
            sccs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def info(self) -> dict:
        return sccs_get_info(self.handle)

    def set_prior(self, prior="normal", variance=1.0):
        sccs_set_prior(self.handle, prior, variance)
        return self

    def fit(self, **kw) -> dict:
        return sccs_fit(self.handle, self.J, **kw)

    def grad_hess(self, j, beta=None):
        return sccs_grad_hess(self.handle, j, beta)

    def logpost(self, beta=None):
        return sccs_logpost(self.handle, beta)

    def heldout_loglik(self, weights=None, beta=None) -> float:
        return sccs_heldout_loglik(self.handle, weights, beta)

    @property
    def beta(self) -> np.ndarray:
        return sccs_get_beta(self.handle, self.J)
