"""GPU parity of the cluster columns: columns with few nonzeros run on one thread-block cluster
(their partial sums meet in distributed shared memory), the others on the whole team, in one
fit.  Every mix is checked against the CPU oracle's Algorithm 1: fixed-cycle trajectories to
1e-11 (Normal prior), converged Laplace fits at the stated bar with the same zero pattern."""
import numpy as np
import pytest

import oracle
from synth import make_dataset, mid_fit_config, paper_scale_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1208_0945_gb300 as P
    return P


def rel(a, b):
    return abs(a - b) / max(1.0, abs(b))


@pytest.mark.parametrize("cluster,cmax", [(16, 500), (16, 5000), (8, 2000), (4, 800), (2, 300), (16, 10**9)])
def test_cluster_and_grid_columns_trajectory(P, cluster, cmax):
    """The 1,000-drug Zipf(1.2) recipe at 2% of its subjects, with the cluster/grid split moved
    across the column sizes (and every column on the cluster in the last case): three cycles
    against the oracle's, beta to 1e-11 and P to 1e-12."""
    d, fit = mid_fit_config(scale=0.02)
    ref = oracle.Problem.from_data(d).fit(prior="normal", variance=fit["variance"], fixed_cycles=3)
    with P.SCCSModel(d, device=0, cluster_ctas=cluster, cluster_max_nnz=cmax) as m:
        info = m.info
        assert info["cluster_ctas"] == cluster
        nnz = np.diff(d.col_ptr)
        assert 0 < info["cluster_columns"] <= d.J
        if cmax < nnz.max():
            assert info["cluster_columns"] < d.J
        m.set_prior("normal", fit["variance"])
        r = m.fit(tol=-1.0, max_cycles=3, history=True)
    assert r["cycles"] == 3
    np.testing.assert_allclose(r["beta"], ref["beta"], atol=1e-11, rtol=0)
    for a, b in zip(r["history"], ref["history"]):
        assert rel(a, b) <= 1e-12
    assert r["nonzero_steps"] == ref["nonzero_steps"]


@pytest.mark.parametrize("cmax", [10**9, 3000])
def test_cluster_columns_converged_laplace(P, cmax):
    """Laplace prior (soft threshold), 5,000 drugs with Zipf(1.1) sizes: every column on the
    cluster, or a split; the converged fit equals the oracle's at the same cycle count with the
    same zero pattern."""
    d, _ = paper_scale_config(scale=0.004)
    orc = oracle.Problem.from_data(d)
    with P.SCCSModel(d, device=0, cluster_ctas=16, cluster_max_nnz=cmax) as m:
        m.set_prior("laplace", 0.05)
        r = m.fit(tol_mode="rel_logpost", tol=1e-13, max_cycles=300)
    assert r["rc"] == 0
    same = orc.fit(prior="laplace", variance=0.05, fixed_cycles=r["cycles"])
    np.testing.assert_allclose(r["beta"], same["beta"], atol=1e-8, rtol=0)
    assert rel(r["logpost"], same["logpost"]) <= 1e-10
    assert np.array_equal(r["beta"] == 0, same["beta"] == 0)
    assert (r["beta"] == 0).any() and (r["beta"] != 0).any()


def test_cluster_on_and_off_agree(P):
    """The same fit with and without cluster columns (same team size): both follow the oracle,
    so they agree to rounding; and a fit repeated on the cluster path is bit for bit the same."""
    d = make_dataset(n_patients=30000, eras=("geometric", 6), J=40, columns=("density_range", 0.0005, 0.2),
                     n_true=5, beta_sd=0.4, seed=31)
    outs = []
    for cl in (16, -1):
        with P.SCCSModel(d, device=0, num_shards=112, cluster_ctas=cl, cluster_max_nnz=4000) as m:
            m.set_prior("normal", 0.3)
            outs.append(m.fit(tol=-1.0, max_cycles=6))
            if cl > 0:
                again = m.fit(tol=-1.0, max_cycles=6)
                assert np.array_equal(again["beta"], outs[0]["beta"]) and again["logpost"] == outs[0]["logpost"]
    np.testing.assert_allclose(outs[0]["beta"], outs[1]["beta"], atol=1e-11, rtol=0)
    ref = oracle.Problem.from_data(d).fit(prior="normal", variance=0.3, fixed_cycles=6)
    np.testing.assert_allclose(outs[0]["beta"], ref["beta"], atol=1e-11, rtol=0)


def test_cluster_options_validated(P):
    d = make_dataset(n_patients=2000, eras=("uniform", 1, 10), J=5, columns=("density", 0.02), n_true=1,
                     beta_sd=0.3, seed=3)
    with pytest.raises(P.SCCSError) as ei:
        P.SCCSModel(d, device=0, cluster_ctas=3)
    assert ei.value.code == P.sccs.E_INVAL
    with pytest.raises(P.SCCSError) as ei:
        P.SCCSModel(d, device=0, num_shards=20, cluster_ctas=16)   # not a multiple of the cluster size
    assert ei.value.code == P.sccs.E_INVAL
    with P.SCCSModel(d, device=0, num_shards=20) as m:              # explicit team: no clusters by default
        assert m.info["cluster_ctas"] == 0 and m.info["cluster_columns"] == 0
    with P.SCCSModel(d, device=0) as m:                             # default team: clusters of 16
        assert m.info["cluster_ctas"] == 16 and m.info["num_shards"] % 16 == 0


def test_cluster_and_grid_columns_without_narrow_columns(P):
    """Every column above the narrow size (so the layout has no narrow arrays), some on the
    cluster and some on the whole team: the grid columns next to cluster runs must not touch the
    narrow path.  Three cycles against the oracle."""
    d = make_dataset(n_patients=60000, eras=("geometric", 8), J=60, columns=("density_range", 0.004, 0.04),
                     n_true=4, beta_sd=0.3, seed=41)
    nnz = np.diff(d.col_ptr)
    assert nnz.min() > 1024
    ref = oracle.Problem.from_data(d).fit(prior="normal", variance=0.5, fixed_cycles=3)
    cmax = int(np.median(nnz))
    with P.SCCSModel(d, device=0, cluster_ctas=16, cluster_max_nnz=cmax) as m:
        info = m.info
        assert info["narrow_columns"] == 0 and 0 < info["cluster_columns"] < d.J
        m.set_prior("normal", 0.5)
        r = m.fit(tol=-1.0, max_cycles=3)
    np.testing.assert_allclose(r["beta"], ref["beta"], atol=1e-11, rtol=0)
    assert rel(r["logpost"], ref["logpost"]) <= 1e-12


def test_tuned_launch_fits_match_the_oracle(P):
    """The launch autotuner's timed probe fits on a dataset, then a fit with the options it chose:
    three cycles against the oracle (every option the tuner can pick gives the oracle's
    trajectory)."""
    from paper_1208_0945_gb300.autotune import tune_launch
    d, fit = mid_fit_config(scale=0.02)
    ch = tune_launch(d, device=0, prior="normal", variance=fit["variance"], cycles=2)
    assert ch.kernel_ms > 0 and len(ch.trials) >= 6
    ref = oracle.Problem.from_data(d).fit(prior="normal", variance=fit["variance"], fixed_cycles=3)
    with P.SCCSModel(d, device=0, **ch.options) as m:
        m.set_prior("normal", fit["variance"])
        r = m.fit(tol=-1.0, max_cycles=3)
    np.testing.assert_allclose(r["beta"], ref["beta"], atol=1e-11, rtol=0)
