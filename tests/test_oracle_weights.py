"""Pins for the oracle's subject weights (Section 2.5: the bootstrap's resampled subjects and
cross-validation's folds), each against a dataset built by hand: a weighted fit must equal an
unweighted fit of the dataset in which subject i appears w_i times, and the held-out predictive
log-likelihood of a fold must equal Eq. 2 on the fold's subjects alone."""
import numpy as np
import pytest

import oracle
from sccs_testlib import input_subjects, random_tiny, replicate_subjects

# The mutation tests swap in a build of the oracle with a planted mistake.
ORACLE_LIB = None


def P(d):
    return oracle.Problem.from_data(d, lib=ORACLE_LIB)


def _data(seed):
    # subjects with n_i = 0 in the input: weights are indexed by input subject, dropped or not
    return random_tiny(seed, n_patients=14, J=4, density=0.4, with_zero_subjects=True, beta_scale=0.4)


@pytest.mark.parametrize("seed", range(3))
def test_unit_weights_are_the_unweighted_fit(seed):
    d = _data(seed)
    p = P(d)
    w = np.ones(p.subjects_in, np.int64)
    a = p.fit(prior="normal", variance=0.5, tol_mode="rel_logpost", tol=1e-14)
    b = p.fit(prior="normal", variance=0.5, tol_mode="rel_logpost", tol=1e-14, weights=w)
    assert np.array_equal(a["beta"], b["beta"]) and a["logpost"] == b["logpost"] and a["cycles"] == b["cycles"]


@pytest.mark.parametrize("seed,prior,var", [(0, "normal", 0.5), (1, "normal", 2.0), (2, "laplace", 0.5),
                                            (3, "none", 1.0)])
def test_weighted_fit_equals_replicated_dataset(seed, prior, var):
    d = _data(seed)
    p = P(d)
    rng = np.random.default_rng(50 + seed)
    w = rng.integers(0, 4, size=p.subjects_in)
    r = P(replicate_subjects(d, w))
    beta = rng.normal(0, 0.5, size=d.J)
    assert p.loglik(beta, weights=w) == pytest.approx(r.loglik(beta), rel=1e-13, abs=1e-12)
    for j in range(d.J):
        gw, hw = p.grad_hess(j, beta, weights=w)
        gr, hr = r.grad_hess(j, beta)
        assert gw == pytest.approx(gr, rel=1e-12, abs=1e-12) and hw == pytest.approx(hr, rel=1e-12, abs=1e-12)
    # at the fixed point (a stopping rule on P can fire a cycle apart on a flat optimum)
    fw = p.fit(prior=prior, variance=var, fixed_cycles=400, weights=w)
    fr = r.fit(prior=prior, variance=var, fixed_cycles=400)
    np.testing.assert_allclose(fw["beta"], fr["beta"], atol=1e-8, rtol=0)
    assert fw["logpost"] == pytest.approx(fr["logpost"], rel=1e-12)


def test_fixed_cycle_trajectory_equals_replicated_dataset():
    """Same Algorithm 1 steps, not just the same fixed point."""
    d = _data(7)
    p = P(d)
    w = np.random.default_rng(7).integers(0, 3, size=p.subjects_in)
    r = P(replicate_subjects(d, w))
    fw = p.fit(prior="normal", variance=1.0, fixed_cycles=3, weights=w)
    fr = r.fit(prior="normal", variance=1.0, fixed_cycles=3)
    np.testing.assert_allclose(fw["beta"], fr["beta"], atol=1e-12, rtol=0)
    np.testing.assert_allclose(fw["history"], fr["history"], rtol=1e-13)


@pytest.mark.parametrize("seed", range(3))
def test_fold_fit_and_heldout_loglik(seed):
    """10-fold cross-validation reading: fit on the other folds (0/1 weights), score Eq. 2 on the
    held-out fold's subjects."""
    d = _data(seed)
    p = P(d)
    rng = np.random.default_rng(90 + seed)
    fold_of = rng.integers(0, 3, size=p.subjects_in)
    for k in range(3):
        train = (fold_of != k).astype(np.int64)
        held = 1 - train
        f = p.fit(prior="normal", variance=0.3, fixed_cycles=300, weights=train)
        sub = P(replicate_subjects(d, train))
        fs = sub.fit(prior="normal", variance=0.3, fixed_cycles=300)
        np.testing.assert_allclose(f["beta"], fs["beta"], atol=1e-8, rtol=0)
        # the held-out fold by itself, as a dataset, at the training fit's beta
        if held.sum() == 0:
            continue
        ho = replicate_subjects(d, held)
        if ho.y.sum() == 0:
            assert p.loglik(f["beta"], weights=held) == 0.0
            continue
        assert p.loglik(f["beta"], weights=held) == pytest.approx(P(ho).loglik(f["beta"]), rel=1e-13, abs=1e-12)


def test_weights_index_input_subjects():
    d = _data(11)
    p = P(d)
    assert p.subjects_in == len(input_subjects(d)) > p.N
