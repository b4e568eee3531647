"""Subject weights on the GPU (Section 2.5: cross-validation folds and bootstrap replicates)
against the oracle, and the fit server's cross-validation and bootstrap requests against the
same calls made one at a time."""
import numpy as np
import pytest

import oracle
from synth import bootstrap_weights, cv_folds, fold_weights, make_dataset, mid_fit_config, tiny_fit_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1208_0945_gb300 as P
    return P


def rel(a, b):
    return abs(a - b) / max(1.0, abs(b))


def _data(n=3000, seed=77, J=30, zero_subjects=True):
    d = make_dataset(n_patients=n, eras=("geometric", 6), J=J, columns=("density_range", 0.01, 0.08),
                     n_true=4, beta_sd=0.5, seed=seed)
    return d


def _n_in(d):
    pid = d.patient_id
    return int(1 + np.count_nonzero(pid[1:] != pid[:-1]))


def test_unit_weights_are_bitwise_the_unweighted_fit(P):
    d, fit = tiny_fit_config()
    with P.SCCSModel(d, device=0, num_shards=4) as m:
        m.set_prior(fit["prior"], fit["variance"])
        a = m.fit(tol=1e-13)
        b = m.fit(tol=1e-13, weights=np.ones(_n_in(d), np.int32))
        c = m.fit(tol=1e-13, precision="fp32_polish", weights=np.ones(_n_in(d), np.int32))
        c0 = m.fit(tol=1e-13, precision="fp32_polish")
    assert np.array_equal(a["beta"], b["beta"]) and a["logpost"] == b["logpost"] and a["cycles"] == b["cycles"]
    assert np.array_equal(c["beta"], c0["beta"]) and c["cycles"] == c0["cycles"]


@pytest.mark.parametrize("prior,var", [("normal", 0.1), ("laplace", 0.2), ("none", 1.0)])
def test_bootstrap_fixed_cycles_against_oracle(P, prior, var):
    d = _data()
    w = bootstrap_weights(_n_in(d), seed=3)
    orc = oracle.Problem.from_data(d)
    ref = orc.fit(prior=prior, variance=var, fixed_cycles=3, weights=w)
    with P.SCCSModel(d, device=0, num_shards=7) as m:
        m.set_prior(prior, var)
        r = m.fit(tol=-1.0, max_cycles=3, weights=w, history=True)
    np.testing.assert_allclose(r["beta"], ref["beta"], atol=1e-11, rtol=0)
    np.testing.assert_allclose(r["history"], ref["history"], rtol=1e-12)


def test_bootstrap_converged_against_oracle(P):
    d = _data(seed=78)
    w = bootstrap_weights(_n_in(d), seed=4)
    ref = oracle.Problem.from_data(d).fit(prior="normal", variance=0.5, fixed_cycles=80, weights=w)
    with P.SCCSModel(d, device=0, num_shards=5) as m:
        m.set_prior("normal", 0.5)
        r = m.fit(tol=1e-15, max_cycles=300, weights=w)
        r32 = m.fit(tol=1e-15, max_cycles=300, weights=w, precision="fp32_polish")
    np.testing.assert_allclose(r["beta"], ref["beta"], atol=1e-8, rtol=0)
    assert rel(r["logpost"], ref["logpost"]) <= 1e-10
    np.testing.assert_allclose(r32["beta"], ref["beta"], atol=1e-6, rtol=0)


def test_cross_validation_fold_fit_and_heldout_loglik(P):
    d = _data(seed=79)
    fold_of = cv_folds(_n_in(d), folds=10, seed=5)
    orc = oracle.Problem.from_data(d)
    with P.SCCSModel(d, device=0, num_shards=6) as m:
        m.set_prior("normal", 0.2)
        for k in (0, 3, 9):
            train, held = fold_weights(fold_of, k)
            r = m.fit(tol=1e-15, max_cycles=300, weights=train)
            ho = m.heldout_loglik(held)
            ref = orc.fit(prior="normal", variance=0.2, fixed_cycles=80, weights=train)
            np.testing.assert_allclose(r["beta"], ref["beta"], atol=1e-8, rtol=0)
            # the evaluation itself, at the GPU's own beta
            assert rel(ho, orc.loglik(r["beta"], weights=held)) <= 1e-12
            # explicit beta, and the plain log-likelihood without weights
            b = np.random.default_rng(k).normal(0, 0.3, d.J)
            assert rel(m.heldout_loglik(held, beta=b), orc.loglik(b, weights=held)) <= 1e-12
            assert rel(m.heldout_loglik(None, beta=b), orc.loglik(b)) <= 1e-12


def test_mid_workload_reduced_scale_weighted(P):
    d, fit = mid_fit_config(scale=0.05)
    w = bootstrap_weights(_n_in(d), seed=6)
    ref = oracle.Problem.from_data(d).fit(prior=fit["prior"], variance=fit["variance"], fixed_cycles=2, weights=w)
    with P.SCCSModel(d, device=0) as m:
        m.set_prior(fit["prior"], fit["variance"])
        r = m.fit(tol=-1.0, max_cycles=2, weights=w)
    np.testing.assert_allclose(r["beta"], ref["beta"], atol=1e-10, rtol=0)
    assert rel(r["logpost"], ref["logpost"]) <= 1e-12


def test_all_zero_weights_and_bad_weights(P):
    d, fit = tiny_fit_config()
    n = _n_in(d)
    with P.SCCSModel(d, device=0, num_shards=3) as m:
        m.set_prior("normal", 1.0)
        r = m.fit(tol=1e-12, weights=np.zeros(n, np.int32))
        assert np.all(r["beta"] == 0.0) and r["logpost"] == 0.0
        bad = np.ones(n, np.int32)
        bad[5] = -1
        with pytest.raises(P.SCCSError) as ei:
            m.fit(weights=bad)
        assert ei.value.code == P.sccs.E_INVAL
        huge = np.full(n, 2**31 - 1, np.int32)
        with pytest.raises(P.SCCSError):
            m.fit(weights=huge)
        with pytest.raises(P.SCCSError):
            m.heldout_loglik(bad)
        # the handle is still usable and unweighted fits are unaffected
        a = m.fit(tol=1e-12)
        ref = oracle.Problem.from_data(d).fit(prior="normal", variance=1.0, fixed_cycles=a["cycles"])
        np.testing.assert_allclose(a["beta"], ref["beta"], atol=1e-11, rtol=0)


def test_server_cv_and_bootstrap_requests_match_one_at_a_time(P):
    """A cross-validation grid (folds x variances) and bootstrap replicates as server requests,
    all in flight together; each equals the same fit + held-out evaluation made alone."""
    datasets = [_data(n=4000, seed=80), _data(n=9000, seed=81, J=45)]
    models = [P.SCCSModel(d, device=0, num_shards=s) for d, s in zip(datasets, (3, 8))]
    try:
        reqs = []
        for di, d in enumerate(datasets):
            n = _n_in(d)
            fold_of = cv_folds(n, folds=10, seed=10 + di)
            for k in (1, 6):
                train, held = fold_weights(fold_of, k)
                for var in (0.05, 0.5):
                    reqs.append((di, "normal", var, train, held, "fp64"))
                reqs.append((di, "laplace", 0.1, train, held, "fp32_polish"))
            for b in range(3):
                reqs.append((di, "normal", 0.2, bootstrap_weights(n, seed=100 * di + b), None, "fp64"))
        alone = []
        for di, prior, var, w, held, prec in reqs:
            m = models[di]
            m.set_prior(prior, var)
            r = m.fit(tol=1e-12, max_cycles=300, weights=w, precision=prec)
            r["heldout_loglik"] = m.heldout_loglik(held) if held is not None else None
            alone.append(r)
        with P.FitServer(device=0, max_inflight=16) as srv:
            tickets = [srv.submit(models[di], prior=prior, variance=var, tol=1e-12, max_cycles=300, weights=w,
                                  heldout_weights=held, precision=prec)
                       for di, prior, var, w, held, prec in reqs]
            got = [srv.wait(t) for t in tickets]
        for g, a, req in zip(got, alone, reqs):
            assert g["status"] == a["status"] and g["cycles"] == a["cycles"]
            assert np.array_equal(g["beta"], a["beta"]) and g["logpost"] == a["logpost"]
            if req[4] is None:
                assert np.isnan(g["heldout_loglik"])
            else:
                assert g["heldout_loglik"] == a["heldout_loglik"]
    finally:
        for m in models:
            m.close()
