"""Helpers shared by the tests: tiny datasets and an independent dense formulation.

The dense formulation writes each subject's conditional likelihood as a multinomial over its
eras with probabilities softmax(log l_ik + x_ik'b) (Eq. 1), and takes the gradient and full
Hessian of that form.  It shares no code with the oracle (which works with the paper's
W = M[L x exp(Xb) x X_j] / M[L x exp(Xb)] ratios) or with the CUDA library.
"""
from __future__ import annotations

import numpy as np

from synth import SCCSData


def from_dense(patient_id, y, L, X) -> SCCSData:
    """Build an SCCSData from dense arrays (X: K x J of 0/1)."""
    X = np.asarray(X)
    K, J = X.shape
    cols = [np.nonzero(X[:, j])[0] for j in range(J)]
    col_ptr = np.zeros(J + 1, np.int64)
    np.cumsum([c.size for c in cols], out=col_ptr[1:])
    row_idx = np.concatenate(cols).astype(np.int32) if J else np.empty(0, np.int32)
    pid = np.asarray(patient_id, np.int64)
    return SCCSData(K=K, N=int(np.unique(pid).size), patient_id=pid,
                    y=np.asarray(y, np.int32), L=np.asarray(L, np.float64), J=J,
                    col_ptr=col_ptr, row_idx=row_idx, beta_true=np.zeros(J), recipe={"name": "dense"})


def to_dense(d: SCCSData) -> np.ndarray:
    X = np.zeros((d.K, d.J))
    for j in range(d.J):
        X[d.column(j), j] = 1.0
    return X


def random_tiny(seed: int, n_patients=12, max_eras=5, J=4, density=0.35, with_zero_subjects=False,
                beta_scale=0.0):
    """A tiny random dataset (dense generation, exact 0/1 design)."""
    rng = np.random.default_rng(seed)
    counts = rng.integers(1, max_eras + 1, size=n_patients)
    pid = np.repeat(np.arange(n_patients), counts)
    K = pid.size
    L = rng.integers(1, 366, size=K).astype(float)
    X = (rng.random((K, J)) < density).astype(float)
    b = rng.normal(0, beta_scale, size=J) if beta_scale > 0 else np.zeros(J)
    lam = L * np.exp(X @ b) / 100.0
    y = rng.poisson(lam)
    for i in range(n_patients):
        rows = np.nonzero(pid == i)[0]
        if y[rows].sum() == 0 and not (with_zero_subjects and i % 3 == 0):
            y[rows[rng.integers(rows.size)]] = 1
    if with_zero_subjects:
        for i in range(0, n_patients, 3):
            y[pid == i] = 0
    return from_dense(pid, y, L, X)


class DenseModel:
    """Independent dense evaluation of the log-posterior, its gradient and Hessian."""

    def __init__(self, d: SCCSData, prior: str = "none", variance: float = 1.0):
        self.X = to_dense(d)
        self.y = d.y.astype(float)
        self.logl = np.log(d.L)
        pid = d.patient_id
        self.groups = [np.nonzero(pid == p)[0] for p in np.unique(pid)]
        self.groups = [g for g in self.groups if self.y[g].sum() > 0]
        self.prior = prior
        self.var = variance

    def _probs(self, beta, g):
        eta = self.logl[g] + self.X[g] @ beta
        m = eta.max()
        w = np.exp(eta - m)
        return w / w.sum(), m + np.log(w.sum())

    def loglik(self, beta):
        tot = 0.0
        for g in self.groups:
            _, lse = self._probs(beta, g)
            n = self.y[g].sum()
            tot += self.y[g] @ (self.X[g] @ beta) - n * lse
        return tot

    def logpost(self, beta):
        lp = self.loglik(beta)
        if self.prior == "normal":
            lp -= beta @ beta / (2 * self.var)
        elif self.prior == "laplace":
            lp -= np.sqrt(2 / self.var) * np.abs(beta).sum()
        return lp

    def grad_hess(self, beta):
        J = self.X.shape[1]
        G = np.zeros(J)
        H = np.zeros((J, J))
        for g in self.groups:
            p, _ = self._probs(beta, g)
            n = self.y[g].sum()
            Xg = self.X[g]
            G += Xg.T @ (self.y[g] - n * p)
            mean = Xg.T @ p
            H -= n * (Xg.T @ (p[:, None] * Xg) - np.outer(mean, mean))
        if self.prior == "normal":
            G -= beta / self.var
            H -= np.eye(J) / self.var
        return G, H

    def newton(self, beta0=None, iters=100, tol=1e-15):
        """Plain multivariate Newton on the smooth log-posterior (no prior or Normal)."""
        J = self.X.shape[1]
        b = np.zeros(J) if beta0 is None else beta0.copy()
        for _ in range(iters):
            G, H = self.grad_hess(b)
            step = np.linalg.solve(H, -G)
            b = b + step
            if np.abs(step).max() < tol:
                break
        return b


def read_golden(path):
    rows, expected = [], []
    section = "data"
    with open(path) as f:
        for line in f:
            s = line.strip()
            if not s:
                continue
            if s.startswith("#"):
                if s.startswith("# expected"):
                    section = "expected"
                continue
            parts = s.split()
            if section == "data":
                rows.append([float(v) for v in parts])
            else:
                expected.append((parts[0], float(parts[1]), float(parts[2])))
    a = np.array(rows)
    pid = a[:, 0].astype(np.int64)
    X = a[:, 2:3]
    return from_dense(pid, a[:, 3].astype(np.int32), a[:, 1], X), expected


def input_subjects(d: SCCSData) -> list:
    """Row ranges of the input subjects (runs of equal patient_id, in input order)."""
    pid = np.asarray(d.patient_id)
    starts = [0] + [k for k in range(1, pid.size) if pid[k] != pid[k - 1]]
    ends = starts[1:] + [pid.size]
    return list(zip(starts, ends))


def replicate_subjects(d: SCCSData, w) -> SCCSData:
    """The dataset in which input subject i appears w[i] times (each copy a subject of its own):
    what a bootstrap resample with multiplicities w, or a fold split with 0/1 weights, is."""
    X = to_dense(d)
    pid, y, L, rows = [], [], [], []
    new_id = 0
    for (a, b), wi in zip(input_subjects(d), w):
        for _ in range(int(wi)):
            pid.extend([new_id] * (b - a))
            y.extend(d.y[a:b])
            L.extend(d.L[a:b])
            rows.append(X[a:b])
            new_id += 1
    Xn = np.concatenate(rows) if rows else np.zeros((0, X.shape[1]))
    return from_dense(np.asarray(pid, np.int64), np.asarray(y), np.asarray(L, float), Xn)
