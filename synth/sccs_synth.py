"""Seeded synthetic self-controlled case series (SCCS) data.

The paper's timings use licensed claims databases (Section 3) that are not available, so
every workload here is synthetic, drawn from the model of Section 2.1:

* subjects i = 1..N, each with K_i eras (constant-exposure intervals); rows of one subject
  are contiguous and subjects appear in increasing id order;
* l_ik: era length in days, integer, uniform on {1..365};
* x_ikj in {0,1}: drug indicators, stored column-wise (CSC, row indices ascending);
* y_ik ~ Poisson(l_ik exp(x_ik' beta_true) / 365), conditioned on n_i = sum_k y_ik >= 1
  (the design keeps cases only, Eq. 1).  The conditioning is sampled exactly: n_i from a
  zero-truncated Poisson, then y_i | n_i ~ Multinomial(n_i, rates / total rate).

Column supports are drawn as Bernoulli(p_j) row processes (geometric skips), so a column's
rows are distinct and sorted.  Column sizes are either a fixed density or a truncated
continuous power law ("Zipf(s) from a to b") by inverse CDF, with column 0 forced to b and
column 1 to a so both extremes exist.

Nothing here evaluates the likelihood, its derivatives or any CCD step.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class SCCSData:
    """One synthetic SCCS dataset in the layout the C ABI takes."""

    K: int                      # rows (eras), including subjects later dropped for n_i = 0
    N: int                      # subjects
    patient_id: np.ndarray      # int64[K], non-decreasing
    y: np.ndarray               # int32[K], event counts
    L: np.ndarray               # float64[K], era lengths (days, integer-valued)
    J: int                      # drug columns
    col_ptr: np.ndarray         # int64[J+1]
    row_idx: np.ndarray         # int32[nnz], ascending within each column
    beta_true: np.ndarray       # float64[J], the generating coefficients
    recipe: dict                # how it was drawn (for reports)

    @property
    def nnz(self) -> int:
        return int(self.col_ptr[-1])

    def column(self, j: int) -> np.ndarray:
        return self.row_idx[self.col_ptr[j]:self.col_ptr[j + 1]]


# --------------------------------------------------------------------------- samplers

def _bernoulli_rows(rng: np.random.Generator, K: int, p: float) -> np.ndarray:
    """Sorted distinct rows of a Bernoulli(p) process on 0..K-1, via geometric gaps."""
    if K <= 0 or p <= 0.0:
        return np.empty(0, dtype=np.int64)
    if p >= 1.0:
        return np.arange(K, dtype=np.int64)
    expected = K * p
    m = int(expected + 6.0 * math.sqrt(expected) + 32)
    gaps = rng.geometric(p, size=m)
    pos = np.cumsum(gaps, dtype=np.int64) - 1
    while pos[-1] < K - 1:
        more = rng.geometric(p, size=max(m // 4, 64))
        pos = np.concatenate([pos, pos[-1] + np.cumsum(more, dtype=np.int64)])
    return pos[pos < K]


def _power_law_sizes(rng: np.random.Generator, J: int, s: float, a: float, b: float) -> np.ndarray:
    """nnz_j i.i.d. from the density proportional to n^-s on [a, b], floored; col 0 = b, col 1 = a."""
    u = rng.random(J)
    if abs(s - 1.0) < 1e-12:
        x = a * np.exp(u * math.log(b / a))
    else:
        e = 1.0 - s
        x = (a ** e + u * (b ** e - a ** e)) ** (1.0 / e)
    sizes = np.floor(x).astype(np.int64)
    if J > 0:
        sizes[0] = int(b)
    if J > 1:
        sizes[1] = int(a)
    return sizes


def _zero_truncated_poisson(rng: np.random.Generator, mu: np.ndarray) -> np.ndarray:
    """Exact draws of Poisson(mu) conditioned on >= 1."""
    n = np.zeros(mu.shape[0], dtype=np.int64)
    big = mu >= 10.0
    ib = np.nonzero(big)[0]
    if ib.size:
        d = rng.poisson(mu[ib])
        zero = d == 0
        while zero.any():                      # P(0) < 5e-5 here: rejection is exact and cheap
            d[zero] = rng.poisson(mu[ib][zero])
            zero = d == 0
        n[ib] = d
    isml = np.nonzero(~big)[0]
    if isml.size:
        m = mu[isml]
        u = rng.random(m.shape[0])
        p0 = np.exp(-m)
        target = p0 + u * (1.0 - p0)           # inverse CDF restricted to k >= 1
        k = np.ones(m.shape[0], dtype=np.int64)
        pk = m * p0
        cdf = p0 + pk
        done = cdf >= target
        it = 0
        while (~done).any() and it < 400:
            nd = ~done
            k[nd] += 1
            pk[nd] *= m[nd] / k[nd]
            cdf[nd] += pk[nd]
            done |= cdf >= target
            it += 1
        n[isml] = k
    return n


def _events_to_rows(rng, mu_k, pat_ptr, n_i):
    """Place n_i events of subject i on its eras with probability proportional to mu_k."""
    K = mu_k.shape[0]
    cum = np.cumsum(mu_k)
    start = pat_ptr[:-1]
    end = pat_ptr[1:]
    base = np.where(start > 0, cum[np.maximum(start - 1, 0)], 0.0)
    tot = cum[end - 1] - base
    ev_pat = np.repeat(np.arange(n_i.shape[0], dtype=np.int64), n_i)
    u = base[ev_pat] + rng.random(ev_pat.shape[0]) * tot[ev_pat]
    r = np.searchsorted(cum, u, side="right")
    r = np.clip(r, start[ev_pat], end[ev_pat] - 1)
    return np.bincount(r, minlength=K).astype(np.int32)


# --------------------------------------------------------------------------- datasets

def make_dataset(*, n_patients: int, eras: tuple, J: int, columns: tuple,
                 n_true: int, beta_sd: float, seed: int, name: str = "custom") -> SCCSData:
    """Draw one dataset.

    eras    = ("uniform", lo, hi) | ("geometric", mean) | ("fixed", k)
    columns = ("density", p) | ("density_range", lo, hi) | ("zipf", s, a, b) | ("sizes", array)
    """
    rng = np.random.default_rng(seed)
    N = int(n_patients)
    kind = eras[0]
    if kind == "uniform":
        counts = rng.integers(int(eras[1]), int(eras[2]) + 1, size=N)
    elif kind == "geometric":
        counts = rng.geometric(1.0 / float(eras[1]), size=N)
    elif kind == "fixed":
        counts = np.full(N, int(eras[1]))
    else:
        raise ValueError(f"unknown era recipe {eras}")
    counts = counts.astype(np.int64)
    K = int(counts.sum())
    pat_ptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(counts, out=pat_ptr[1:])
    patient_id = np.repeat(np.arange(N, dtype=np.int64), counts)
    L = rng.integers(1, 366, size=K).astype(np.float64)

    ckind = columns[0]
    if ckind == "density":
        probs = np.full(J, float(columns[1]))
    elif ckind == "densities":                      # one density per column (shared across datasets)
        probs = np.asarray(columns[1], dtype=np.float64)
        assert probs.shape == (J,)
    elif ckind == "density_range":
        probs = rng.uniform(float(columns[1]), float(columns[2]), size=J)
    elif ckind == "zipf":
        sizes = _power_law_sizes(rng, J, float(columns[1]), float(columns[2]), float(columns[3]))
        probs = np.minimum(1.0, sizes / max(K, 1))
    elif ckind == "sizes":
        sizes = np.asarray(columns[1], dtype=np.int64)
        assert sizes.shape[0] == J
        probs = np.minimum(1.0, sizes / max(K, 1))
    else:
        raise ValueError(f"unknown column recipe {columns}")
    cols = [_bernoulli_rows(rng, K, float(p)) for p in probs]
    col_ptr = np.zeros(J + 1, dtype=np.int64)
    np.cumsum([c.shape[0] for c in cols], out=col_ptr[1:])
    row_idx = (np.concatenate(cols) if cols else np.empty(0, np.int64)).astype(np.int32)

    beta_true = np.zeros(J)
    if n_true > 0 and J > 0:
        which = rng.choice(J, size=min(n_true, J), replace=False)
        beta_true[which] = rng.normal(0.0, beta_sd, size=which.shape[0])
    xb = np.zeros(K)
    for j in np.nonzero(beta_true)[0]:
        xb[cols[j]] += beta_true[j]
    mu_k = L * np.exp(xb) / 365.0
    mu_i = np.add.reduceat(mu_k, pat_ptr[:-1]) if N > 0 else np.zeros(0)
    n_i = _zero_truncated_poisson(rng, mu_i)
    y = _events_to_rows(rng, mu_k, pat_ptr, n_i)
    recipe = dict(name=name, seed=seed, n_patients=N, eras=list(eras), J=J,
                  columns=[c if not isinstance(c, np.ndarray) else "explicit" for c in columns],
                  n_true=n_true, beta_sd=beta_sd, K=K, nnz=int(col_ptr[-1]))
    return SCCSData(K=K, N=N, patient_id=patient_id, y=y, L=L, J=J, col_ptr=col_ptr,
                    row_idx=row_idx, beta_true=beta_true, recipe=recipe)


def tiny_fit_config(seed: int = 1208) -> tuple[SCCSData, dict]:
    """2,000 subjects, 1-10 eras each, 50 drugs at 2% density, 5 true effects ~ N(0, 0.3^2).

    Fit: Normal prior with variance 1, FP64, stop when |delta log-posterior| < 1e-10.
    """
    d = make_dataset(n_patients=2000, eras=("uniform", 1, 10), J=50, columns=("density", 0.02),
                     n_true=5, beta_sd=0.3, seed=seed, name="tiny-2k-subjects-50-drugs")
    fit = dict(prior="normal", variance=1.0, tol_mode="abs_logpost", tol=1e-10, max_cycles=1000)
    return d, fit


def mid_fit_config(seed: int = 1209, scale: float = 1.0) -> tuple[SCCSData, dict]:
    """1M subjects (~10M eras, geometric mean 10), 1,000 drugs with Zipf(1.2) sizes 10..2M.

    20 true effects ~ N(0, 0.5^2); Normal prior variance 0.1; FP64.  `scale` shrinks the
    subject count and the largest column together (for parity tests at reduced size).
    """
    n = max(int(round(1_000_000 * scale)), 100)
    b = max(2_000_000 * scale, 20.0)
    d = make_dataset(n_patients=n, eras=("geometric", 10), J=1000, columns=("zipf", 1.2, 10, b),
                     n_true=20, beta_sd=0.5, seed=seed,
                     name=f"mid-{n}-subjects-1000-drugs-zipf1.2")
    fit = dict(prior="normal", variance=0.1, tol_mode="rel_logpost", tol=1e-12, max_cycles=1000)
    return d, fit


def large_columns_config(seed: int = 1215, scale: float = 1.0) -> tuple[SCCSData, dict]:
    """1M subjects (eras geometric, mean 10), 16 drug columns of 1M to 2M nonzeros each (uniform
    sizes), 5 true effects N(0, 0.3^2); Normal prior variance 0.1; a fixed 4 cycles per fit."""
    n = max(1000, int(round(1_000_000 * scale)))
    rng = np.random.default_rng(seed)
    sizes = (rng.integers(1_000_000, 2_000_001, size=16) * (n / 1_000_000)).astype(np.int64)
    d = make_dataset(n_patients=n, eras=("geometric", 10), J=16, columns=("sizes", sizes), n_true=5, beta_sd=0.3,
                     seed=seed, name="large-columns")
    return d, {"prior": "normal", "variance": 0.1, "cycles": 4}


def paper_scale_config(seed: int = 1210, scale: float = 1.0) -> tuple[SCCSData, dict]:
    """4M subjects (~40M eras), 5,000 drugs with Zipf(1.1) sizes 10..5M, 50 true effects.

    Laplace prior variance 0.05.
    """
    n = max(int(round(4_000_000 * scale)), 100)
    b = max(5_000_000 * scale, 20.0)
    d = make_dataset(n_patients=n, eras=("geometric", 10), J=5000, columns=("zipf", 1.1, 10, b),
                     n_true=50, beta_sd=0.5, seed=seed,
                     name=f"paper-scale-{n}-subjects-5000-drugs-zipf1.1")
    fit = dict(prior="laplace", variance=0.05, tol_mode="rel_logpost", tol=1e-12, max_cycles=1000)
    return d, fit


def batched_fit_configs(n_fits: int = 64, min_subjects: int = 2000, max_subjects: int = 100_000,
                        J: int = 500, seed: int = 1211) -> list:
    """Independent fits for a batched launch: subjects per fit log-uniform in
    [min_subjects, max_subjects], eras geometric with mean 8, J binary drugs whose densities
    (uniform 0.5-5%) are shared by all fits while the rows are drawn per fit, 3 true effects
    per fit, Normal prior variance 0.01 / 0.1 / 1 in turn."""
    plan = batched_fit_plan(n_fits, min_subjects, max_subjects, J, seed)
    return [batched_fit_one(plan, f) for f in range(n_fits)]


def batched_fit_plan(n_fits: int = 256, min_subjects: int = 2000, max_subjects: int = 500_000, J: int = 500,
                     seed: int = 1211) -> dict:
    """What batched_fit_one needs to draw fit f of a batch on its own (for parallel drawing)."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(min_subjects), np.log(max_subjects), size=n_fits)).astype(int)
    dens = rng.uniform(0.005, 0.05, size=J)
    return dict(sizes=sizes, dens=dens, J=J, seed=seed)


def batched_fit_one(plan: dict, f: int):
    """Fit f of a batch: the same draw as batched_fit_configs gives for f."""
    d = make_dataset(n_patients=int(plan["sizes"][f]), eras=("geometric", 8), J=plan["J"],
                     columns=("densities", plan["dens"]), n_true=3, beta_sd=0.5, seed=plan["seed"] * 1000 + f,
                     name=f"batched-fit-{f}")
    fit = dict(prior="normal", variance=(0.01, 0.1, 1.0)[f % 3], tol_mode="rel_logpost", tol=1e-12,
               max_cycles=1000)
    return d, fit


PRIOR_VARIANCE_GRID = (0.01, 0.02, 0.05, 0.1, 0.2, 0.5, 1.0)


def serving_pool_plan(n_outcomes: int = 32, min_eras: int = 20_000, max_eras: int = 20_000_000,
                      min_drugs: int = 1000, max_drugs: int = 5000, seed: int = 1212) -> dict:
    """Outcomes a fit server holds: eras log-uniform in [min_eras, max_eras] (subjects = eras / 10,
    geometric eras with mean 10), drugs uniform in [min_drugs, max_drugs], columns drawn like
    the 1M-subject workload's (Zipf(1.2) sizes from 10 up to eras / 5)."""
    rng = np.random.default_rng(seed)
    eras = np.exp(rng.uniform(np.log(min_eras), np.log(max_eras), size=n_outcomes))
    drugs = rng.integers(min_drugs, max_drugs + 1, size=n_outcomes)
    return dict(eras=eras, drugs=drugs, seed=seed)


def serving_outcome(plan: dict, o: int) -> SCCSData:
    K = float(plan["eras"][o])
    n = max(int(round(K / 10.0)), 100)
    b = max(K / 5.0, 20.0)
    return make_dataset(n_patients=n, eras=("geometric", 10), J=int(plan["drugs"][o]), columns=("zipf", 1.2, 10, b),
                        n_true=20, beta_sd=0.5, seed=plan["seed"] * 1000 + o, name=f"served-outcome-{o}")


def serving_requests(n_requests: int, rate_per_s: float, n_outcomes: int, seed: int = 1213, folds: int = 0) -> list:
    """Poisson arrivals at `rate_per_s`: (arrival time s, outcome, prior, variance, fold) with the
    prior Normal or Laplace at even odds and the variance drawn from PRIOR_VARIANCE_GRID; fold is
    uniform in 1..folds (0 when folds = 0, a fit on all subjects)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n_requests))
    out = []
    for k in range(n_requests):
        out.append((float(t[k]), int(rng.integers(n_outcomes)), "normal" if rng.random() < 0.5 else "laplace",
                    float(PRIOR_VARIANCE_GRID[rng.integers(len(PRIOR_VARIANCE_GRID))]),
                    int(rng.integers(1, folds + 1)) if folds > 0 else 0))
    return out


def cv_folds(n_subjects: int, folds: int = 10, seed: int = 1214) -> np.ndarray:
    """Section 2.5's random split of the subjects into `folds` portions of (nearly) equal size:
    the fold index 0..folds-1 of each input subject."""
    rng = np.random.default_rng(seed)
    fold_of = np.empty(n_subjects, np.int32)
    fold_of[rng.permutation(n_subjects)] = np.arange(n_subjects) % folds
    return fold_of


def fold_weights(fold_of: np.ndarray, k: int) -> tuple:
    """(training weights, held-out weights) for fold k: 1 off the fold and 1 on it."""
    held = (fold_of == k).astype(np.int32)
    return (1 - held).astype(np.int32), held


def bootstrap_weights(n_subjects: int, seed: int) -> np.ndarray:
    """One non-parametric bootstrap replicate of the subjects (Section 2.5): how many times each
    input subject is drawn when n_subjects are drawn with replacement."""
    rng = np.random.default_rng(seed)
    return rng.multinomial(n_subjects, np.full(n_subjects, 1.0 / n_subjects)).astype(np.int32)


CONFIGS = {
    "tiny": tiny_fit_config,
    "mid": mid_fit_config,
    "paper": paper_scale_config,
}
