"""Pins for the CPU oracle: each test checks it against something other than itself.

* Eq. 2 against scipy's multinomial and Poisson log-pmfs (the conditional and the profiled
  Poisson forms of the SCCS likelihood).
* Eqs. 7-9 against central finite differences of Eq. 2.
* Algorithm 1's fixed point against closed forms (golden fixture), a 1-D bounded minimiser,
  full multivariate Newton on an independent dense formulation, and KKT certificates.
* Invariants: monotone ascent, dropping n_i = 0 subjects, merging duplicate eras,
  column permutation, additivity over subject shards.
"""
import math
import os

import numpy as np
import pytest
import scipy.optimize
import scipy.stats
from scipy.special import gammaln

import oracle
from sccs_testlib import DenseModel, from_dense, random_tiny, read_golden, to_dense

HERE = os.path.dirname(os.path.abspath(__file__))

# The mutation tests swap in a build of the oracle with a planted mistake.
ORACLE_LIB = None


def P(d):
    return oracle.Problem.from_data(d, lib=ORACLE_LIB)


# ----------------------------------------------------------------------------- Eq. 2

@pytest.mark.parametrize("seed", range(6))
def test_loglik_equals_conditional_multinomial(seed):
    """Eq. 1 says y_i | n_i is multinomial over the eras with p_ik proportional to l_ik e^{x_ik'b}.
    Eq. 2 is its log-pmf minus the constants log n_i! - sum log y_ik! + sum y_ik log l_ik."""
    d = random_tiny(seed, n_patients=10, J=3, beta_scale=0.5)
    p = P(d)
    X = to_dense(d)
    rng = np.random.default_rng(100 + seed)
    for _ in range(3):
        beta = rng.normal(0, 0.7, size=d.J)
        eta = X @ beta
        ref = 0.0
        for i in np.unique(d.patient_id):
            g = np.nonzero(d.patient_id == i)[0]
            yi = d.y[g]
            n = int(yi.sum())
            if n == 0:
                continue
            w = d.L[g] * np.exp(eta[g])
            lp = scipy.stats.multinomial.logpmf(yi, n, w / w.sum())
            ref += lp - gammaln(n + 1) + gammaln(yi + 1).sum() - (yi * np.log(d.L[g])).sum()
        assert p.loglik(beta) == pytest.approx(ref, rel=1e-11, abs=1e-9)


@pytest.mark.parametrize("seed", range(4))
def test_loglik_equals_profiled_poisson(seed):
    """The SCCS likelihood is the Poisson likelihood with each subject's intercept phi_i
    maximised out (Section 2.1: the subject effect is conditioned away).  The profile is
    taken numerically here, with scipy's Poisson log-pmf."""
    d = random_tiny(seed, n_patients=6, J=2, beta_scale=0.4)
    p = P(d)
    X = to_dense(d)
    beta = np.random.default_rng(seed).normal(0, 0.5, size=d.J)
    eta = X @ beta
    total = 0.0
    for i in np.unique(d.patient_id):
        g = np.nonzero(d.patient_id == i)[0]
        yi, n = d.y[g], int(d.y[g].sum())
        if n == 0:
            continue
        f = lambda phi: -scipy.stats.poisson.logpmf(yi, d.L[g] * np.exp(phi + eta[g])).sum()
        res = scipy.optimize.minimize_scalar(f, bracket=(-12.0, 2.0), tol=1e-14)
        prof = -res.fun
        # remove the constants the conditional form drops: n log n - n + sum y log l - sum log y!
        total += prof - (n * math.log(n) - n + (yi * np.log(d.L[g])).sum() - gammaln(yi + 1).sum())
    assert p.loglik(beta) == pytest.approx(total, rel=1e-9, abs=1e-7)


# ----------------------------------------------------------------------------- Eqs. 7-9

def _fd(f, x, h):
    return (f(x + h) - f(x - h)) / (2 * h), (f(x + h) - 2 * f(x) + f(x - h)) / (h * h)


@pytest.mark.parametrize("seed", range(5))
def test_grad_hess_finite_differences(seed):
    """g_j, h_j (Eqs. 7-9) equal the first and second derivatives of Eq. 2 along e_j
    (central differences with one Richardson extrapolation)."""
    d = random_tiny(seed, n_patients=15, J=5, density=0.4, beta_scale=0.5)
    p = P(d)
    rng = np.random.default_rng(7 + seed)
    beta = rng.normal(0, 0.6, size=d.J)
    for j in range(d.J):
        def f(t):
            b = beta.copy()
            b[j] = t
            return p.loglik(b)
        h0 = 1e-3
        g1, h1 = _fd(f, beta[j], h0)
        g2, h2 = _fd(f, beta[j], h0 / 2)
        g_fd = (4 * g2 - g1) / 3
        h_fd = (4 * h2 - h1) / 3
        g, h = p.grad_hess(j, beta)
        assert g == pytest.approx(g_fd, rel=1e-7, abs=1e-7)
        assert h == pytest.approx(h_fd, rel=1e-5, abs=1e-5)
        assert h <= 0.0


def test_grad_hess_against_dense_softmax_form():
    """Diagonal of the dense softmax-form Hessian and its gradient equal Eqs. 7-9."""
    d = random_tiny(3, n_patients=20, J=6, density=0.3, beta_scale=0.5)
    p = P(d)
    m = DenseModel(d)
    beta = np.random.default_rng(1).normal(0, 0.5, size=d.J)
    G, H = m.grad_hess(beta)
    for j in range(d.J):
        g, h = p.grad_hess(j, beta)
        assert g == pytest.approx(G[j], rel=1e-12, abs=1e-11)
        assert h == pytest.approx(H[j, j], rel=1e-12, abs=1e-11)


def test_grad_hess_at_zero_exact_rationals():
    """At b = 0 (Algorithm 1's start) W_i is a ratio of integer era lengths, so g_j and h_j
    are rationals; compare with exact fraction arithmetic."""
    from fractions import Fraction
    d = random_tiny(11, n_patients=9, J=3, density=0.5)
    p = P(d)
    for j in range(d.J):
        inX = np.zeros(d.K, bool)
        inX[d.column(j)] = True
        G, H = Fraction(0), Fraction(0)
        for i in np.unique(d.patient_id):
            g = np.nonzero(d.patient_id == i)[0]
            n = int(d.y[g].sum())
            if n == 0:
                continue
            den = sum(Fraction(int(v)) for v in d.L[g])
            num = sum(Fraction(int(v)) for v in d.L[g][inX[g]])
            W = num / den
            G += n * W
            H += n * W * (1 - W)
        ytx = int(d.y[inX].sum())
        g, h = p.grad_hess(j, np.zeros(d.J))
        assert g == pytest.approx(float(ytx - G), rel=1e-14, abs=1e-13)
        assert h == pytest.approx(float(-H), rel=1e-14, abs=1e-13)


# ----------------------------------------------------------------------------- Algorithm 1

def test_golden_one_covariate_closed_forms():
    d, expected = read_golden(os.path.join(HERE, "golden", "one_covariate_closed_form.txt"))
    p = P(d)
    for prior, var, b_expected in expected:
        r = p.fit(prior=prior, variance=var if var > 0 else 1.0, tol_mode="abs_logpost", tol=1e-15,
                  max_cycles=500)
        assert r["beta"][0] == pytest.approx(b_expected, abs=1e-9), (prior, var)
        if b_expected == 0.0:
            assert r["beta"][0] == 0.0  # the soft threshold keeps it exactly at zero


def test_golden_trust_region_trajectory():
    """The Genkin trust region (R1): on a one-drug example whose Newton step has a closed form,
    the first two steps are cut to the radius (b = 1, then b = 3) and the radius update
    T <- max(2|db|, T/2) decides the second cut; the later cycles follow the closed form."""
    d, expected = read_golden(os.path.join(HERE, "golden", "one_covariate_trust_trajectory.txt"))
    p = P(d)
    for _tag, cycle, b_expected in expected:
        r = p.fit(prior="none", fixed_cycles=int(cycle))
        assert r["cycles"] == int(cycle)
        if b_expected in (1.0, 3.0):
            assert r["beta"][0] == b_expected, cycle        # a clamp to the radius is exact
        else:
            assert r["beta"][0] == pytest.approx(b_expected, rel=0, abs=1e-12), cycle
    # the limit is the closed-form MLE log(A / (n - A)) - log r = log 100
    r = p.fit(prior="none", tol_mode="abs_logpost", tol=1e-15, max_cycles=100)
    assert r["beta"][0] == pytest.approx(math.log(100.0), abs=1e-12)


@pytest.mark.parametrize("seed", [2, 5])
def test_genkin_xbeta_stopping_rule(seed):
    """Genkin's X-beta rule (R4, after the Section 2.2 criterion): a fit stops after the first
    cycle t with sum_k |(Xb_t - Xb_{t-1})_k| / (1 + sum_k |(Xb_t)_k|) < tol.  The statistic is
    computed here from a dense X and the oracle's beta after each cycle, and the tolerance is
    placed where the rule without the 1 + in the denominator would stop one cycle later."""
    d = random_tiny(seed, n_patients=8, max_eras=3, J=3, density=0.3, beta_scale=0.3)
    p = P(d)
    X = to_dense(d)
    T = 6
    betas = [np.zeros(d.J)] + [p.fit(prior="normal", variance=1.0, fixed_cycles=t)["beta"] for t in range(1, T + 1)]
    xb = [X @ b for b in betas]
    stat = [None] + [np.abs(xb[t] - xb[t - 1]).sum() / (1.0 + np.abs(xb[t]).sum()) for t in range(1, T + 1)]
    asum = [None] + [np.abs(xb[t]).sum() for t in range(1, T + 1)]
    t_star = 3
    assert stat[t_star] > 0 and stat[t_star - 1] > stat[t_star] * 1.5, stat
    tol = stat[t_star] * (1.0 + 0.5 / asum[t_star])
    # the rule without the 1 + would not stop at t_star
    assert np.abs(xb[t_star] - xb[t_star - 1]).sum() / asum[t_star] > tol
    r = p.fit(prior="normal", variance=1.0, tol_mode="genkin_xbeta", tol=tol, max_cycles=50)
    assert r["status"] == oracle.OK and r["cycles"] == t_star, (r["cycles"], stat, tol)
    np.testing.assert_array_equal(r["beta"], betas[t_star])


def test_column_covering_whole_subjects_q_zero():
    """R5: a column holding every era of each subject it touches has W_i = 1 for those subjects,
    so g_j = Y'X_j - sum n_i = 0 and h_j = 0 exactly (Eqs. 7-9).  The 1-D optimum of the
    penalised objective along that coordinate is then b_j = 0: the Laplace step returns to 0
    (cut to the trust radius 1 first when |b_j| > 1), the Normal step -b_j (s2/s2) lands on 0
    up to rounding, and without a prior the step is 0."""
    pid = [0, 0, 0, 1, 1, 2, 2, 2, 3, 3]
    L = [30.0, 40.0, 50.0, 20.0, 60.0, 10.0, 70.0, 90.0, 25.0, 35.0]
    y = [1, 0, 2, 1, 1, 0, 1, 1, 2, 0]
    X = np.zeros((10, 2))
    X[[0, 1, 2, 5, 6, 7], 0] = 1.0          # subjects 0 and 2, all their eras
    X[[1, 3, 8], 1] = 1.0
    d = from_dense(pid, y, L, X)
    p = P(d)
    g, h = p.grad_hess(0, np.array([0.4, -0.3]))
    assert g == 0.0 and h == 0.0
    # Laplace, |b| > radius: cut to the radius, then to 0
    r = p.fit(prior="laplace", variance=0.5, beta0=np.array([1.7, 0.0]), fixed_cycles=1)
    assert r["beta"][0] == pytest.approx(0.7, abs=1e-15)
    r = p.fit(prior="laplace", variance=0.5, beta0=np.array([1.7, 0.0]), fixed_cycles=2)
    assert r["beta"][0] == 0.0
    r = p.fit(prior="laplace", variance=0.5, beta0=np.array([-0.6, 0.0]), fixed_cycles=1)
    assert r["beta"][0] == 0.0
    r = p.fit(prior="normal", variance=0.3, beta0=np.array([0.6, 0.0]), fixed_cycles=1)
    assert abs(r["beta"][0]) < 1e-15
    r = p.fit(prior="none", beta0=np.array([0.6, 0.0]), fixed_cycles=1)
    assert r["beta"][0] == 0.6 and not r["warning"]


@pytest.mark.parametrize("r_ratio", [0.1, 0.5, 2.0])
def test_one_covariate_closed_form_random(r_ratio):
    """b_hat = log(A / (n - A)) - log r when every subject has exposed/unexposed time ratio r."""
    rng = np.random.default_rng(int(r_ratio * 10))
    pid, y, L, X = [], [], [], []
    for i in range(30):
        u = float(rng.integers(10, 200))
        yu, ye = rng.integers(0, 4), rng.integers(0, 4)
        if yu + ye == 0:
            ye = 1
        pid += [i, i]
        L += [u, u * r_ratio]
        y += [yu, ye]
        X += [[0.0], [1.0]]
    d = from_dense(pid, y, L, np.array(X))
    A = sum(y[1::2])
    n = sum(y)
    expected = math.log(A / (n - A)) - math.log(r_ratio)
    r = P(d).fit(prior="none", tol_mode="abs_logpost", tol=1e-15, max_cycles=500)
    assert r["beta"][0] == pytest.approx(expected, abs=1e-9)


@pytest.mark.parametrize("seed", range(3))
def test_one_covariate_general_minimiser(seed):
    """A single drug with a Normal prior: Algorithm 1 agrees with a bounded 1-D minimiser of
    the (pinned) log-posterior."""
    d = random_tiny(seed, n_patients=40, J=1, density=0.4, beta_scale=0.8)
    p = P(d)
    var = 0.7
    f = lambda b: -p.logpost(np.array([b]), "normal", var)
    res = scipy.optimize.minimize_scalar(f, bounds=(-10, 10), method="bounded",
                                         options={"xatol": 1e-12})
    r = p.fit(prior="normal", variance=var, tol_mode="abs_logpost", tol=1e-15, max_cycles=500)
    assert r["beta"][0] == pytest.approx(res.x, abs=1e-6)
    g, h = p.grad_hess(0, r["beta"])
    assert abs(g - r["beta"][0] / var) < 1e-9


@pytest.mark.parametrize("seed,prior", [(0, "none"), (1, "normal"), (2, "normal"), (3, "none")])
def test_ccd_matches_multivariate_newton(seed, prior):
    """The CCD fixed point equals full Newton on the dense softmax formulation (J <= 6)."""
    d = random_tiny(seed, n_patients=60, max_eras=6, J=5, density=0.35, beta_scale=0.6)
    var = 0.5
    m = DenseModel(d, prior=prior, variance=var)
    b_newton = m.newton()
    r = P(d).fit(prior=prior, variance=var, tol_mode="abs_logpost",
                                        tol=1e-14, max_cycles=5000)
    assert r["status"] == oracle.OK
    np.testing.assert_allclose(r["beta"], b_newton, atol=1e-9, rtol=0)
    assert r["logpost"] == pytest.approx(m.logpost(b_newton), rel=1e-12)


@pytest.mark.parametrize("seed,var", [(0, 0.05), (1, 0.2), (2, 1.0)])
def test_laplace_kkt_certificate(seed, var):
    """At the Laplace MAP: b_j != 0 => g_j = lambda sign(b_j); b_j = 0 => |g_j| <= lambda,
    with g_j from the dense formulation (independent of the oracle)."""
    d = random_tiny(seed, n_patients=80, max_eras=6, J=6, density=0.3, beta_scale=0.7)
    lam = math.sqrt(2 / var)
    r = P(d).fit(prior="laplace", variance=var, tol_mode="abs_logpost",
                                        tol=1e-15, max_cycles=5000)
    G, _ = DenseModel(d).grad_hess(r["beta"])
    assert (r["beta"] != 0).any()
    for j in range(d.J):
        if r["beta"][j] != 0.0:
            # a stop on |dP| < 1e-15 leaves |db| ~ sqrt(dP / q): residuals of order 1e-7
            assert abs(G[j] - lam * np.sign(r["beta"][j])) < 1e-6, j
        else:
            assert abs(G[j]) <= lam + 1e-9, j


@pytest.mark.parametrize("prior,var", [("normal", 1.0), ("laplace", 0.1), ("none", 1.0)])
def test_monotone_ascent(prior, var):
    from synth import tiny_fit_config
    d, _ = tiny_fit_config()
    r = P(d).fit(prior=prior, variance=var, tol_mode="abs_logpost",
                                        tol=1e-12, max_cycles=200)
    h = r["history"]
    assert np.all(np.diff(h) >= -1e-13 * np.abs(h[1:]) - 1e-12)


def test_zero_event_subjects_contribute_nothing():
    """Section 2.1: subjects with n_i = 0 drop out; results are bitwise unchanged."""
    d0 = random_tiny(5, n_patients=30, J=4, with_zero_subjects=True, beta_scale=0.3)
    keep = np.ones(d0.K, bool)
    for i in np.unique(d0.patient_id):
        g = d0.patient_id == i
        if d0.y[g].sum() == 0:
            keep[g] = False
    X = to_dense(d0)
    d1 = from_dense(d0.patient_id[keep], d0.y[keep], d0.L[keep], X[keep])
    p0, p1 = P(d0), P(d1)
    assert p0.dropped_patients > 0 and p1.dropped_patients == 0
    r0 = p0.fit(prior="normal", variance=0.5, tol=1e-13)
    r1 = p1.fit(prior="normal", variance=0.5, tol=1e-13)
    assert np.array_equal(r0["beta"], r1["beta"])
    assert r0["logpost"] == r1["logpost"]


def test_merging_duplicate_eras_leaves_likelihood_unchanged():
    """Eras are unique exposure patterns within a subject (Section 2.3): two eras with the
    same pattern merge into one with summed length and events without changing Eq. 2."""
    pid = [0, 0, 0, 1, 1]
    X = np.array([[1, 0], [1, 0], [0, 1], [0, 0], [1, 1]], float)
    L = [10.0, 30.0, 5.0, 7.0, 11.0]
    y = [1, 2, 0, 1, 1]
    d = from_dense(pid, y, L, X)
    dm = from_dense([0, 0, 1, 1], [3, 0, 1, 1], [40.0, 5.0, 7.0, 11.0], X[[0, 2, 3, 4]])
    p, pm = P(d), P(dm)
    for beta in ([0.3, -0.2], [1.5, 0.7], [-2.0, 0.1]):
        b = np.array(beta)
        assert p.loglik(b) == pytest.approx(pm.loglik(b), rel=1e-14)


def test_map_invariant_to_column_order():
    d = random_tiny(9, n_patients=50, J=5, density=0.3, beta_scale=0.5)
    perm = np.array([3, 0, 4, 2, 1])
    X = to_dense(d)
    dp = from_dense(d.patient_id, d.y, d.L, X[:, perm])
    r = P(d).fit(prior="normal", variance=0.3, tol=1e-14, max_cycles=5000)
    rp = P(dp).fit(prior="normal", variance=0.3, tol=1e-14, max_cycles=5000)
    np.testing.assert_allclose(rp["beta"], r["beta"][perm], atol=1e-9)


def test_subject_shards_add_up():
    """L, g_j and h_j are sums over subjects (M is block diagonal), so subject shards add up.
    This is the decomposition a subject-sharded step relies on."""
    d = random_tiny(4, n_patients=40, J=3, beta_scale=0.5)
    X = to_dense(d)
    beta = np.array([0.2, -0.4, 0.7])
    full = P(d)
    cut = d.patient_id < 17
    parts = [P(from_dense(d.patient_id[m], d.y[m], d.L[m], X[m])) for m in (cut, ~cut)]
    assert full.loglik(beta) == pytest.approx(sum(q.loglik(beta) for q in parts), rel=1e-13)
    for j in range(3):
        g, h = full.grad_hess(j, beta)
        gs = [q.grad_hess(j, beta) for q in parts]
        assert g == pytest.approx(sum(x[0] for x in gs), rel=1e-12, abs=1e-12)
        assert h == pytest.approx(sum(x[1] for x in gs), rel=1e-12, abs=1e-12)


def test_input_validation():
    d = random_tiny(0)
    with pytest.raises(oracle.OracleError):
        oracle.Problem(d.K, d.patient_id[::-1].copy(), d.y, d.L, d.J, d.col_ptr, d.row_idx)
    bad = d.row_idx.copy()
    bad[0] = d.K
    with pytest.raises(oracle.OracleError):
        oracle.Problem(d.K, d.patient_id, d.y, d.L, d.J, d.col_ptr, bad)


@pytest.mark.parametrize("seed", range(4))
def test_raw_eval_equals_canonical_oracle(seed):
    """The evaluation straight from the input arrays (used for sampled checks at sizes too big
    for the canonical copy) against the canonical oracle, with zero-event subjects and rows of
    a column in shuffled order."""
    d = random_tiny(seed, n_patients=25, J=5, with_zero_subjects=True, beta_scale=0.5)
    rng = np.random.default_rng(seed)
    for j in range(d.J):            # shuffle each column's rows
        a, b = d.col_ptr[j], d.col_ptr[j + 1]
        d.row_idx[a:b] = rng.permutation(d.row_idx[a:b])
    beta = rng.normal(0, 0.6, size=d.J)
    p = oracle.Problem.from_data(d, lib=ORACLE_LIB)
    ll, g, h = oracle.raw_eval(d, beta, np.arange(d.J), lib=ORACLE_LIB)
    assert ll == pytest.approx(p.loglik(beta), rel=1e-13, abs=1e-12)
    for j in range(d.J):
        gc, hc = p.grad_hess(j, beta)
        assert g[j] == pytest.approx(gc, rel=1e-12, abs=1e-12) and h[j] == pytest.approx(hc, rel=1e-12, abs=1e-12)
