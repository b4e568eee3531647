"""Cross-validation and bootstrap through the package's resampling API (Section 2.5), on the GPU
through the fit server, against the oracle: every replicate's or fold's MAP against the
oracle's Algorithm 1 run with the same weights for the same number of cycles, the held-out
predictive log-likelihood against the oracle's Eq. 2 at that MAP, and the summaries (quantile
intervals, non-zero fractions, the chosen variance) against the same summaries of the oracle's
results."""
import numpy as np
import pytest

import oracle
from synth import bootstrap_weights, cv_folds, make_dataset

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__._build_module().build()
    import paper_1208_0945_gb300 as P
    return P


def _data(n, seed, J=25):
    return make_dataset(n_patients=n, eras=("geometric", 6), J=J, columns=("density_range", 0.01, 0.1),
                        n_true=5, beta_sd=0.6, seed=seed)


def _n_in(d):
    pid = d.patient_id
    return int(1 + np.count_nonzero(pid[1:] != pid[:-1]))


def test_bootstrap_intervals_against_oracle(P):
    from paper_1208_0945_gb300 import resampling
    d = _data(3000, 90)
    orc = oracle.Problem.from_data(d)
    n = _n_in(d)
    W = np.stack([bootstrap_weights(n, seed=500 + b) for b in range(24)])
    with P.SCCSModel(d, device=0, num_shards=4) as m:
        assert resampling.subjects_in(m) == n
        out = resampling.bootstrap(m, "laplace", 0.1, weights=W, tol=1e-13, max_cycles=500)
    assert out["not_converged"] == 0 and out["replicates"].shape == (24, d.J)
    ref = np.stack([orc.fit(prior="laplace", variance=0.1, fixed_cycles=int(c), weights=w)["beta"]
                    for c, w in zip(out["cycles"], W)])
    np.testing.assert_allclose(out["replicates"], ref, atol=1e-8, rtol=0)
    assert np.array_equal(out["replicates"] == 0, ref == 0)
    full = orc.fit(prior="laplace", variance=0.1, fixed_cycles=int(out["cycles_hat"]))["beta"]
    np.testing.assert_allclose(out["beta_hat"], full, atol=1e-8, rtol=0)
    s = resampling.interval_summary(ref)
    np.testing.assert_allclose(out["lower"], s["lower"], atol=1e-8, rtol=0)
    np.testing.assert_allclose(out["upper"], s["upper"], atol=1e-8, rtol=0)
    assert np.array_equal(out["p_nonzero"], s["p_nonzero"])
    # the intervals are non-trivial: some coefficients are zero in some replicates only
    assert ((out["p_nonzero"] > 0) & (out["p_nonzero"] < 1)).any()
    assert np.all(out["lower"] <= out["upper"])


def test_cross_validation_against_oracle(P):
    from paper_1208_0945_gb300 import resampling
    d = _data(4000, 91)
    orc = oracle.Problem.from_data(d)
    n = _n_in(d)
    fold_of = cv_folds(n, folds=5, seed=3)
    variances = (0.003, 0.05, 1.0)
    with P.SCCSModel(d, device=0, num_shards=6) as m:
        out = resampling.cross_validate(m, "normal", variances, fold_of=fold_of, tol=1e-13, max_cycles=500)
    assert out["heldout"].shape == (3, 5)
    ref = np.empty((3, 5))
    for vi, v in enumerate(variances):
        for ki, k in enumerate(out["folds"]):
            train = (fold_of != k).astype(np.int64)
            held = (fold_of == k).astype(np.int64)
            r = orc.fit(prior="normal", variance=v, fixed_cycles=int(out["cycles"][vi, ki]), weights=train)
            np.testing.assert_allclose(out["betas"][vi, ki], r["beta"], atol=1e-8, rtol=0)
            ref[vi, ki] = orc.loglik(r["beta"], weights=held)
    np.testing.assert_allclose(out["heldout"], ref, rtol=1e-10)
    assert out["best_variance"] == variances[int(np.argmax(ref.mean(axis=1)))]
    np.testing.assert_allclose(out["mean_heldout"], ref.mean(axis=1), rtol=1e-10)


def test_resampling_with_drawn_weights_and_a_shared_server(P):
    """Weights drawn from a seed (twice the same), requests through a caller's server."""
    from paper_1208_0945_gb300 import resampling
    d = _data(2500, 92, J=15)
    with P.SCCSModel(d, device=0, num_shards=4) as m, P.FitServer(device=0, max_inflight=8) as srv:
        a = resampling.bootstrap(m, "normal", 0.5, replicates=6, seed=11, server=srv)
        b = resampling.bootstrap(m, "normal", 0.5, replicates=6, seed=11, server=srv)
        cv = resampling.cross_validate(m, "normal", (0.1, 1.0), folds=4, seed=5, server=srv)
    assert np.array_equal(a["replicates"], b["replicates"])
    assert a["replicates"].shape == (6, d.J) and np.isfinite(cv["heldout"]).all()
    assert cv["best_variance"] in (0.1, 1.0)
