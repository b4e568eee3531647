"""Cross-validation and the non-parametric bootstrap over the fit server (Section 2.5).

Both are many weighted fits of one resident dataset: a fold's training fit counts the subjects
of the other folds once and its own zero times, and evaluates the predictive log-likelihood of
Eq. 2 on the held-out fold at the fold's MAP; a bootstrap replicate counts each subject as many
times as a resample of the subjects with replacement drew it.  Every fit runs on the GPU through
the library's fit server (continuous batching of the requests in flight); this module only
draws the weights (or takes them as given), submits the requests and summarises the results:

* `bootstrap` returns, per coefficient, the (1 - level)/2 and (1 + level)/2 quantiles of its
  replicate MAP estimates -- the paper's 95% intervals from the 2.5% and 97.5% quantiles -- and
  p_hat_j, the fraction of replicates in which beta_j is not zero (under the Laplace prior the
  paper's stand-in for the posterior probability of a non-zero effect);
* `cross_validate` returns the held-out predictive log-likelihood of every (variance, fold)
  pair, its mean over the folds per variance, and the variance with the largest mean.

Weights are indexed by input subject (runs of equal patient id in the arrays the dataset was
created from, subjects without events included).  When not given they are drawn from `seed`
with NumPy's PCG64 generator: a fold per subject from a random permutation cut into near-equal
parts, and a replicate's multiplicities from a multinomial(n, 1/n) draw.
"""
from __future__ import annotations

import numpy as np

from .sccs import FitServer


def subjects_in(model) -> int:
    """Input subjects of a resident dataset (the length of a weight vector)."""
    return int(model.info["subjects_in"])


def draw_folds(n_subjects: int, folds: int, seed: int) -> np.ndarray:
    """Fold number (1..folds) per input subject: a random permutation cut into near-equal parts."""
    if folds < 2 or folds > n_subjects:
        raise ValueError("need 2 <= folds <= subjects")
    perm = np.random.default_rng(seed).permutation(n_subjects)
    fold_of = np.empty(n_subjects, np.int64)
    fold_of[perm] = np.arange(n_subjects) % folds + 1
    return fold_of


def draw_bootstrap(n_subjects: int, replicates: int, seed: int) -> np.ndarray:
    """(replicates, n_subjects) multiplicities, each row one resample with replacement."""
    rng = np.random.default_rng(seed)
    return rng.multinomial(n_subjects, np.full(n_subjects, 1.0 / n_subjects), size=replicates).astype(np.int32)


def interval_summary(betas: np.ndarray, level: float = 0.95) -> dict:
    """Quantile intervals and the non-zero fraction of replicate estimates (replicates x J)."""
    b = np.asarray(betas, np.float64)
    if b.ndim != 2 or b.shape[0] < 1:
        raise ValueError("betas must be (replicates, J) with at least one replicate")
    if not 0.0 < level < 1.0:
        raise ValueError("level must be in (0, 1)")
    lo, hi = np.quantile(b, [(1.0 - level) / 2.0, (1.0 + level) / 2.0], axis=0)
    return {"lower": lo, "upper": hi, "p_nonzero": np.mean(b != 0.0, axis=0)}


def _run(model, requests, server, alt, max_inflight, window: int = 1024):
    """Submit every request (at most `window` outstanding, well inside the server's host queue)
    and return the results in request order."""
    own = server is None
    srv = FitServer(device=model.device, max_inflight=max_inflight) if own else server
    try:
        results = [None] * len(requests)
        pending = []                     # (request index, ticket), oldest first
        for i, kw in enumerate(requests):
            if len(pending) >= window:
                k, t = pending.pop(0)
                results[k] = srv.wait(t)
            pending.append((i, srv.submit(model, alt=alt, **kw)))
        for k, t in pending:
            results[k] = srv.wait(t)
        return results
    finally:
        if own:
            srv.close()


def _check_done(results, what):
    bad = [r["status"] for r in results if r["status"] not in (0, 1)]
    if bad:
        raise RuntimeError(f"{len(bad)} {what} fits failed (status {sorted(set(bad))})")


def bootstrap(model, prior: str, variance: float, *, replicates: int = 200, seed: int = 0, weights=None,
              level: float = 0.95, tol_mode: str = "rel_logpost", tol: float = 1e-12, max_cycles: int = 1000,
              precision: str = "fp64", server: FitServer | None = None, alt=None, max_inflight: int = 64) -> dict:
    """Non-parametric bootstrap of the MAP estimate: `replicates` weighted fits (or one per row
    of `weights`), the full-data fit, and their summary (see the module docstring).  Results
    with status NOT_CONVERGED (max_cycles reached) are kept and counted in `not_converged`."""
    n = subjects_in(model)
    W = draw_bootstrap(n, replicates, seed) if weights is None else np.ascontiguousarray(weights, np.int32)
    if W.ndim != 2 or W.shape[1] != n or W.shape[0] < 1:
        raise ValueError(f"weights must be (replicates, {n})")
    common = dict(prior=prior, variance=variance, tol_mode=tol_mode, tol=tol, max_cycles=max_cycles,
                  precision=precision)
    reqs = [dict(common)] + [dict(common, weights=w) for w in W]
    res = _run(model, reqs, server, alt, max_inflight)
    _check_done(res, "bootstrap")
    betas = np.stack([r["beta"] for r in res[1:]])
    out = {"beta_hat": res[0]["beta"], "logpost_hat": res[0]["logpost"], "cycles_hat": res[0]["cycles"],
           "replicates": betas, "cycles": np.array([r["cycles"] for r in res[1:]]),
           "not_converged": int(sum(r["status"] == 1 for r in res))}
    out.update(interval_summary(betas, level))
    return out


def cross_validate(model, prior: str, variances, *, folds: int = 10, seed: int = 0, fold_of=None,
                   tol_mode: str = "rel_logpost", tol: float = 1e-12, max_cycles: int = 1000,
                   precision: str = "fp64", server: FitServer | None = None, alt=None,
                   max_inflight: int = 64) -> dict:
    """K-fold cross-validation of the prior variance: for each variance and fold, the MAP on the
    other folds and Eq. 2's log-likelihood of the held-out fold at that MAP; the best variance
    has the largest mean held-out log-likelihood."""
    n = subjects_in(model)
    f = draw_folds(n, folds, seed) if fold_of is None else np.ascontiguousarray(fold_of, np.int64)
    if f.shape != (n,):
        raise ValueError(f"fold_of must have one entry per input subject ({n})")
    ks = np.unique(f)
    if ks.size < 2:
        raise ValueError("need at least two folds")
    vs = [float(v) for v in variances]
    if not vs:
        raise ValueError("no variances")
    reqs = []
    for v in vs:
        for k in ks:
            train = (f != k).astype(np.int32)
            held = (f == k).astype(np.int32)
            reqs.append(dict(prior=prior, variance=v, tol_mode=tol_mode, tol=tol, max_cycles=max_cycles,
                             precision=precision, weights=train, heldout_weights=held))
    res = _run(model, reqs, server, alt, max_inflight)
    _check_done(res, "cross-validation")
    H = np.array([r["heldout_loglik"] for r in res], np.float64).reshape(len(vs), ks.size)
    mean = H.mean(axis=1)
    return {"variances": np.array(vs), "folds": ks, "heldout": H, "mean_heldout": mean,
            "best_variance": vs[int(np.argmax(mean))],
            "betas": np.stack([r["beta"] for r in res]).reshape(len(vs), ks.size, -1),
            "cycles": np.array([r["cycles"] for r in res]).reshape(len(vs), ks.size)}
