"""Serial FP64 CPU oracle for the BSCCS cyclic-coordinate-descent MAP fit (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use
this package.  It shares no code with the CUDA library: the C source in this directory is
compiled on its own with gcc and loaded with ctypes.  The product path never imports it.

Functions follow the paper (Suchard et al., arXiv 1208.0945):
  loglik      Eq. 2, evaluated directly from its definition
  logpost     Eq. 2 plus the log prior of Eq. 3 with every constant dropped
  grad_hess   Eqs. 7-9 from scratch at a given beta (log-likelihood derivatives only)
  fit         Algorithm 1 with the Newton step of Eq. 4, a Genkin trust region and the
              Section 2.3 sparse updates of Xb, L x exp(Xb) and M[L x exp(Xb)]
  weights=    (loglik, grad_hess, fit) Section 2.5's resampling: subject i counted w_i times,
              the bootstrap's multiplicities or a cross-validation fold's 0/1 mask; the
              held-out predictive log-likelihood is loglik with the fold's mask
Readings of points the paper leaves open are listed at the top of ``sccs_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sccs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsccs_oracle.so")
_lock = threading.Lock()
_lib = None

PRIOR = {"none": 0, "normal": 1, "laplace": 2}
TOL = {"abs_logpost": 0, "rel_logpost": 1, "genkin_xbeta": 2}
OK, NOT_CONVERGED = 0, 1


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


def compile_command(src: str, out: str) -> list:
    return ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
            src, "-o", out, "-lm"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math, no vectorisation flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = compile_command(_SRC, tmp)
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    """Declare the C signatures on a loaded oracle library."""
    P = ctypes.c_void_p
    i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
    lib.oracle_create.restype = P
    lib.oracle_create.argtypes = [ctypes.c_int64, i64p, i32p, f64p, ctypes.c_int32, i64p, i32p,
                                  ctypes.POINTER(ctypes.c_int)]
    lib.oracle_free.argtypes = [P]
    lib.oracle_dims.argtypes = [P, i64p]
    lib.oracle_loglik.restype = ctypes.c_double
    lib.oracle_loglik.argtypes = [P, f64p]
    lib.oracle_logpost.restype = ctypes.c_double
    lib.oracle_logpost.argtypes = [P, f64p, ctypes.c_int, ctypes.c_double]
    lib.oracle_grad_hess.restype = ctypes.c_int
    lib.oracle_grad_hess.argtypes = [P, f64p, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]
    lib.oracle_fit.restype = ctypes.c_int
    lib.oracle_fit.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                               ctypes.c_int, P, f64p, f64p, ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int)]
    lib.oracle_raw_eval.restype = ctypes.c_int
    lib.oracle_raw_eval.argtypes = [ctypes.c_int64, i64p, i32p, f64p, ctypes.c_int32, i64p, i32p, f64p,
                                    ctypes.c_int32, i32p, ctypes.POINTER(ctypes.c_double), f64p, f64p]
    lib.oracle_subjects_in.restype = ctypes.c_int64
    lib.oracle_subjects_in.argtypes = [P]
    lib.oracle_loglik_w.restype = ctypes.c_double
    lib.oracle_loglik_w.argtypes = [P, f64p, P]
    lib.oracle_grad_hess_w.restype = ctypes.c_int
    lib.oracle_grad_hess_w.argtypes = [P, f64p, ctypes.c_int32, P, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]
    lib.oracle_fit_w.restype = ctypes.c_int
    lib.oracle_fit_w.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                 ctypes.c_int, P, P, f64p, f64p, ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int)]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
        return _lib


def load_variant(so_path: str):
    """Load another build of the oracle source (used by the tests that plant mistakes)."""
    return _bind(ctypes.CDLL(so_path))


class Problem:
    """A canonicalised SCCS problem held by the C oracle (subjects with n_i = 0 removed)."""

    def __init__(self, K, patient_id, y, L, J, col_ptr, row_idx, lib=None):
        lib = _load() if lib is None else lib
        self._lib = lib
        self._keep = [np.ascontiguousarray(patient_id, np.int64), np.ascontiguousarray(y, np.int32),
                      np.ascontiguousarray(L, np.float64), np.ascontiguousarray(col_ptr, np.int64),
                      np.ascontiguousarray(row_idx, np.int32)]
        err = ctypes.c_int(0)
        pid, yy, LL, cp, ri = self._keep
        self._p = lib.oracle_create(int(K), pid, yy, LL, int(J), cp, ri, ctypes.byref(err))
        if not self._p:
            raise OracleError(err.value, "create")
        dims = np.zeros(6, np.int64)
        lib.oracle_dims(self._p, dims)
        self.K, self.N, self.J, self.nnz, self.dropped_patients, self.dropped_rows = (int(v) for v in dims)
        self.subjects_in = int(lib.oracle_subjects_in(self._p))

    @classmethod
    def from_data(cls, d, lib=None) -> "Problem":
        return cls(d.K, d.patient_id, d.y, d.L, d.J, d.col_ptr, d.row_idx, lib=lib)

    def __del__(self):
        p = getattr(self, "_p", None)
        if p:
            self._lib.oracle_free(p)
            self._p = None

    def _beta(self, beta):
        b = np.zeros(self.J) if beta is None else np.ascontiguousarray(beta, np.float64)
        assert b.shape == (self.J,)
        return b

    def _w(self, weights):
        """Subject weights (R9), one non-negative integer per input subject; None = all 1."""
        if weights is None:
            return None, None
        w = np.ascontiguousarray(weights, np.int64)
        assert w.shape == (self.subjects_in,) and (w >= 0).all()
        return w, w.ctypes.data

    def loglik(self, beta=None, weights=None) -> float:
        if weights is not None:
            w, wp = self._w(weights)
            return float(self._lib.oracle_loglik_w(self._p, self._beta(beta), wp))
        return float(self._lib.oracle_loglik(self._p, self._beta(beta)))

    def logpost(self, beta=None, prior="normal", variance=1.0) -> float:
        return float(self._lib.oracle_logpost(self._p, self._beta(beta), PRIOR[prior], float(variance)))

    def grad_hess(self, j: int, beta=None, weights=None) -> tuple[float, float]:
        g, h = ctypes.c_double(), ctypes.c_double()
        if weights is not None:
            w, wp = self._w(weights)
            rc = self._lib.oracle_grad_hess_w(self._p, self._beta(beta), int(j), wp, ctypes.byref(g),
                                              ctypes.byref(h))
        else:
            rc = self._lib.oracle_grad_hess(self._p, self._beta(beta), int(j), ctypes.byref(g), ctypes.byref(h))
        if rc != OK:
            raise OracleError(rc, "grad_hess")
        return g.value, h.value

    def fit(self, prior="normal", variance=1.0, tol_mode="abs_logpost", tol=1e-10,
            max_cycles=1000, beta0=None, fixed_cycles: int | None = None, weights=None) -> dict:
        """Algorithm 1.  fixed_cycles=T runs exactly T cycles (no convergence test); weights (R9)
        count subject i w_i times (per input subject; None = all 1)."""
        if fixed_cycles is not None:
            max_cycles, tol = int(fixed_cycles), -1.0
        beta = np.zeros(self.J)
        hist = np.full(max_cycles + 1, np.nan)
        cyc = ctypes.c_int(0)
        nz = ctypes.c_int64(0)
        warn = ctypes.c_int(0)
        b0 = None
        if beta0 is not None:
            b0 = np.ascontiguousarray(beta0, np.float64)
            assert b0.shape == (self.J,)
        if weights is not None:
            w, wp = self._w(weights)
            rc = self._lib.oracle_fit_w(self._p, PRIOR[prior], float(variance), TOL[tol_mode], float(tol),
                                        int(max_cycles), None if b0 is None else b0.ctypes.data, wp, beta, hist,
                                        ctypes.byref(cyc), ctypes.byref(nz), ctypes.byref(warn))
        else:
            rc = self._lib.oracle_fit(self._p, PRIOR[prior], float(variance), TOL[tol_mode], float(tol),
                                      int(max_cycles), None if b0 is None else b0.ctypes.data, beta, hist,
                                      ctypes.byref(cyc), ctypes.byref(nz), ctypes.byref(warn))
        if rc < 0:
            raise OracleError(rc, "fit")
        t = cyc.value
        return dict(status=rc, beta=beta, cycles=t, logpost=float(hist[t]), history=hist[:t + 1].copy(),
                    nonzero_steps=int(nz.value), warning=bool(warn.value))


def raw_eval(d, beta, cols, lib=None):
    """Eq. 2 and (g_j, h_j) of Eqs. 7-9 for the columns `cols`, straight from the input arrays of
    dataset d (no canonical copy; for sampled checks of very large problems).
    Returns (loglik, g array, h array)."""
    lib = _load() if lib is None else lib
    cols = np.ascontiguousarray(cols, np.int32)
    g = np.zeros(cols.size)
    h = np.zeros(cols.size)
    ll = ctypes.c_double()
    rc = lib.oracle_raw_eval(int(d.K), np.ascontiguousarray(d.patient_id, np.int64),
                             np.ascontiguousarray(d.y, np.int32), np.ascontiguousarray(d.L, np.float64), int(d.J),
                             np.ascontiguousarray(d.col_ptr, np.int64), np.ascontiguousarray(d.row_idx, np.int32),
                             np.ascontiguousarray(beta, np.float64), int(cols.size), cols, ctypes.byref(ll), g, h)
    if rc != OK:
        raise OracleError(rc, "raw_eval")
    return ll.value, g, h
