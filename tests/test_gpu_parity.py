"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element by element.

Tolerances (FP64 path):
  g_j, h_j                      relative 1e-12 (both sides sum the same terms in FP64; the
                                orders differ, so a few ulps of each of ~1e3 terms)
  fixed-cycle trajectories      |d beta| <= 1e-11, relative d P <= 1e-12 (Normal prior)
  converged fits                |d beta| <= 1e-8, relative d P <= 1e-10 (the stated bar)
"""
import numpy as np
import pytest

import oracle
from sccs_testlib import from_dense, random_tiny, to_dense
from synth import make_dataset, mid_fit_config, paper_scale_config, tiny_fit_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1208_0945_gb300 as P
    return P


def gpu_model(P, d, **kw):
    return P.SCCSModel(d, device=0, **kw)


def rel(a, b):
    return abs(a - b) / max(1.0, abs(b))


def check_grad_hess(P, d, betas, columns=None, **kw):
    orc = oracle.Problem.from_data(d)
    with gpu_model(P, d, **kw) as m:
        for beta in betas:
            for j in (range(d.J) if columns is None else columns):
                g, h = m.grad_hess(j, beta)
                go, ho = orc.grad_hess(j, beta)
                scale_g = max(1.0, abs(go))
                assert abs(g - go) <= 1e-12 * scale_g + 1e-12 * abs(ho), (j, g, go)
                assert abs(h - ho) <= 1e-12 * max(1.0, abs(ho)), (j, h, ho)


def test_grad_hess_tiny_config(P):
    d, _ = tiny_fit_config()
    rng = np.random.default_rng(0)
    check_grad_hess(P, d, [np.zeros(d.J), rng.normal(0, 0.3, d.J)])


@pytest.mark.parametrize("shards,threads", [(1, 64), (7, 128), (64, 512), (0, 256)])
def test_grad_hess_across_launch_shapes(P, shards, threads):
    """Several tiles per slice and ragged tails: 30k subjects, columns from 0.1% to 30% density."""
    d = make_dataset(n_patients=30000, eras=("geometric", 6), J=12, columns=("density_range", 0.001, 0.3),
                     n_true=4, beta_sd=0.4, seed=77)
    rng = np.random.default_rng(1)
    check_grad_hess(P, d, [rng.normal(0, 0.4, d.J)], num_shards=shards, threads_per_block=threads)


def test_logpost_matches_oracle(P):
    d, _ = tiny_fit_config()
    orc = oracle.Problem.from_data(d)
    rng = np.random.default_rng(3)
    with gpu_model(P, d) as m:
        for prior, var in (("none", 1.0), ("normal", 0.5), ("laplace", 0.2)):
            m.set_prior(prior, var)
            for _ in range(3):
                b = rng.normal(0, 0.5, d.J)
                lp, ll = m.logpost(b)
                assert rel(ll, orc.loglik(b)) <= 1e-12
                assert rel(lp, orc.logpost(b, prior, var)) <= 1e-12


@pytest.mark.parametrize("prior,var", [("normal", 1.0), ("normal", 0.1), ("none", 1.0)])
def test_fixed_cycle_trajectory(P, prior, var):
    d, _ = tiny_fit_config()
    ref = oracle.Problem.from_data(d).fit(prior=prior, variance=var, fixed_cycles=3)
    with gpu_model(P, d) as m:
        m.set_prior(prior, var)
        r = m.fit(tol=-1.0, max_cycles=3, history=True)
    assert r["cycles"] == 3
    np.testing.assert_allclose(r["beta"], ref["beta"], atol=1e-11, rtol=0)
    for a, b in zip(r["history"], ref["history"]):
        assert rel(a, b) <= 1e-12
    assert r["nonzero_steps"] == ref["nonzero_steps"]


def check_stop(ref_hist, cycles, tol_mode, tol, P_scale):
    """The GPU stopped where the oracle's own trajectory meets the stopping rule, up to the
    rounding of |dP| (a few ulps of |P|): a cycle-count difference of one at the threshold is
    rounding, not a different algorithm."""
    slack = 64 * np.finfo(float).eps * P_scale
    dP = np.abs(np.diff(ref_hist))
    if tol_mode == "rel_logpost":
        dP = dP / np.maximum(1.0, np.abs(ref_hist[1:]))
        slack /= max(1.0, P_scale)
    assert dP[cycles - 1] < tol + slack
    if cycles >= 2:
        assert dP[cycles - 2] >= tol - slack


def compare_converged(r, orc, prior, var, tol_mode, tol, atol=1e-8, rtol_p=1e-10):
    """A converged GPU fit against the oracle's Algorithm 1 run for the same number of cycles
    (the two trajectories agree to rounding), and the stop checked on the oracle's trajectory."""
    ref = orc.fit(prior=prior, variance=var, fixed_cycles=r["cycles"] + 1)
    same = orc.fit(prior=prior, variance=var, fixed_cycles=r["cycles"])
    np.testing.assert_allclose(r["beta"], same["beta"], atol=atol, rtol=0)
    assert rel(r["logpost"], same["logpost"]) <= rtol_p
    check_stop(ref["history"], r["cycles"], tol_mode, tol, abs(ref["logpost"]))
    return same


def test_converged_tiny_config(P):
    """The tiny workload with its own stopping rule (|dP| < 1e-10): the GPU fit equals the
    oracle's trajectory at the same cycle count, and stops where the oracle's trajectory meets
    the rule; then both are run to a tight stop and compared at the stated bar."""
    d, fit = tiny_fit_config()
    orc = oracle.Problem.from_data(d)
    with gpu_model(P, d) as m:
        m.set_prior(fit["prior"], fit["variance"])
        r = m.fit(tol_mode=fit["tol_mode"], tol=fit["tol"], max_cycles=fit["max_cycles"], history=True)
        tight = m.fit(tol_mode="rel_logpost", tol=1e-15, max_cycles=200)
    assert r["rc"] == 0
    ref = orc.fit(prior=fit["prior"], variance=fit["variance"], fixed_cycles=r["cycles"] + 1)
    same = orc.fit(prior=fit["prior"], variance=fit["variance"], fixed_cycles=r["cycles"])
    np.testing.assert_allclose(r["beta"], same["beta"], atol=1e-11, rtol=0)
    assert rel(r["logpost"], same["logpost"]) <= 1e-12
    check_stop(ref["history"], r["cycles"], fit["tol_mode"], fit["tol"], abs(ref["logpost"]))
    h = r["history"]
    assert np.all(np.diff(h) >= -1e-13 * np.abs(h[1:]) - 1e-12)  # monotone ascent
    assert tight["rc"] == 0
    compare_converged(tight, orc, fit["prior"], fit["variance"], "rel_logpost", 1e-15)


@pytest.mark.parametrize("var", [0.05, 0.5])
def test_converged_laplace(P, var):
    """Laplace prior: soft-threshold decisions may flip transiently near |g| = lambda, so
    only converged results are compared (tight stop on both sides)."""
    d, _ = paper_scale_config(scale=0.004)  # 16k subjects, 5000 drugs, Zipf(1.1) sizes
    orc = oracle.Problem.from_data(d)
    with gpu_model(P, d) as m:
        m.set_prior("laplace", var)
        r = m.fit(tol_mode="rel_logpost", tol=1e-13, max_cycles=300)
    assert r["rc"] == 0
    same = compare_converged(r, orc, "laplace", var, "rel_logpost", 1e-13)
    assert np.array_equal(r["beta"] == 0, same["beta"] == 0)
    assert (r["beta"] == 0).any() and (r["beta"] != 0).any()


def test_mid_config_reduced_scale(P):
    """The 1,000-drug Zipf(1.2) recipe at 2% of its subjects: trajectories and converged fit."""
    d, fit = mid_fit_config(scale=0.02)
    orc = oracle.Problem.from_data(d)
    ref3 = orc.fit(prior="normal", variance=fit["variance"], fixed_cycles=2)
    with gpu_model(P, d) as m:
        m.set_prior("normal", fit["variance"])
        r3 = m.fit(tol=-1.0, max_cycles=2)
        r = m.fit(tol_mode="rel_logpost", tol=1e-14, max_cycles=200)
    np.testing.assert_allclose(r3["beta"], ref3["beta"], atol=1e-11, rtol=0)
    assert r["rc"] == 0
    compare_converged(r, orc, "normal", fit["variance"], "rel_logpost", 1e-14)


def test_full_mid_config_as_benchmarked(P):
    """The benchmarked workload (1M subjects, ~10M eras, 1,000 drugs) in the bench's launch
    shape: the whole fit against the oracle's, plus sampled g_j at the fitted beta."""
    d, fit = mid_fit_config()
    orc = oracle.Problem.from_data(d)
    with gpu_model(P, d) as m:
        m.set_prior("normal", fit["variance"])
        r = m.fit(tol_mode=fit["tol_mode"], tol=fit["tol"], max_cycles=fit["max_cycles"])
        assert r["rc"] == 0
        ref = compare_converged(r, orc, "normal", fit["variance"], fit["tol_mode"], fit["tol"])
        for j in (0, 1, 2, 500, 999):
            g, h = m.grad_hess(j, ref["beta"])
            go, ho = orc.grad_hess(j, ref["beta"])
            assert abs(g - go) <= 1e-10 * max(1.0, abs(ho)), j
            assert rel(h, ho) <= 1e-11, j


def test_repeat_fits_are_bitwise_identical(P):
    d, _ = mid_fit_config(scale=0.01)
    with gpu_model(P, d) as m:
        m.set_prior("normal", 0.1)
        a = m.fit(tol=1e-13)
        b = m.fit(tol=1e-13)
    assert np.array_equal(a["beta"], b["beta"]) and a["logpost"] == b["logpost"]


def test_results_do_not_depend_on_launch_shape(P):
    d = make_dataset(n_patients=20000, eras=("geometric", 8), J=30, columns=("density_range", 0.005, 0.1),
                     n_true=5, beta_sd=0.5, seed=5)
    outs = []
    for shards, threads in ((0, 512), (13, 96), (1, 64)):
        with gpu_model(P, d, num_shards=shards, threads_per_block=threads) as m:
            m.set_prior("normal", 0.3)
            outs.append(m.fit(tol=-1.0, max_cycles=8))
    for o in outs[1:]:
        np.testing.assert_allclose(o["beta"], outs[0]["beta"], atol=1e-10, rtol=0)


def test_warm_start_and_beta0(P):
    d, _ = tiny_fit_config()
    orc = oracle.Problem.from_data(d)
    b0 = np.random.default_rng(9).normal(0, 0.2, d.J)
    ref = orc.fit(prior="normal", variance=0.4, beta0=b0, fixed_cycles=2)
    with gpu_model(P, d) as m:
        m.set_prior("normal", 0.4)
        r = m.fit(beta0=b0, tol=-1.0, max_cycles=2)
        np.testing.assert_allclose(r["beta"], ref["beta"], atol=1e-11, rtol=0)
        # warm start continues from the previous fit
        ref2 = orc.fit(prior="normal", variance=0.4, beta0=ref["beta"], fixed_cycles=1)
        r2 = m.fit(warm_start=True, tol=-1.0, max_cycles=1)
        np.testing.assert_allclose(r2["beta"], ref2["beta"], atol=1e-11, rtol=0)
        np.testing.assert_allclose(m.beta, r2["beta"], atol=0, rtol=0)


# ------------------------------------------------------------------ edge cases

def test_edge_empty_columns_and_zero_event_subjects(P):
    d0 = random_tiny(2, n_patients=40, J=5, density=0.3, with_zero_subjects=True, beta_scale=0.4)
    X = to_dense(d0)
    X[:, 2] = 0.0                                  # an empty column
    d = from_dense(d0.patient_id, d0.y, d0.L, X)
    orc = oracle.Problem.from_data(d)
    with gpu_model(P, d) as m:
        info = m.info
        assert info["subjects_in"] - info["subjects_kept"] > 0
        m.set_prior("normal", 0.7)
        r = m.fit(tol_mode="abs_logpost", tol=1e-12, max_cycles=500)
    assert r["beta"][2] == 0.0
    compare_converged(r, orc, "normal", 0.7, "abs_logpost", 1e-12)


def test_edge_column_covering_whole_subjects(P):
    """W_i = 1 for every touched subject: h_j = 0 and g_j = 0 (flat direction)."""
    pid = np.repeat(np.arange(6), 3)
    X = np.zeros((18, 2))
    X[0:3, 0] = 1.0      # all eras of subject 0
    X[6:9, 0] = 1.0      # all eras of subject 2
    X[1::3, 1] = 1.0
    y = np.tile([1, 0, 2], 6)
    d = from_dense(pid, y, np.arange(1, 19, dtype=float), X)
    orc = oracle.Problem.from_data(d)
    with gpu_model(P, d) as m:
        g, h = m.grad_hess(0, np.array([0.3, -0.2]))
        go, ho = orc.grad_hess(0, np.array([0.3, -0.2]))
        assert abs(h) <= 1e-14 and abs(g) <= 1e-12
        assert abs(g - go) <= 1e-12 and abs(h - ho) <= 1e-12
        m.set_prior("laplace", 0.5)
        r = m.fit(tol_mode="abs_logpost", tol=1e-12, max_cycles=200)
    assert r["beta"][0] == 0.0
    compare_converged(r, orc, "laplace", 0.5, "abs_logpost", 1e-12)


def test_edge_single_subject_and_single_column(P):
    pid = np.zeros(4, np.int64)
    X = np.array([[1.0], [0.0], [1.0], [0.0]])
    d = from_dense(pid, [2, 1, 0, 1], [10.0, 20.0, 30.0, 40.0], X)
    orc = oracle.Problem.from_data(d)
    with gpu_model(P, d) as m:
        r = m.fit(tol_mode="abs_logpost", tol=1e-15, max_cycles=300)
    ref = orc.fit(prior="none", fixed_cycles=r["cycles"])
    np.testing.assert_allclose(r["beta"], ref["beta"], atol=1e-11)
    # closed form: A = 2 exposed events of n = 4, exposed time 40 vs unexposed 60
    assert r["beta"][0] == pytest.approx(np.log(2 / 2) - np.log(40 / 60), abs=1e-9)


def test_edge_duplicate_rows_rejected(P):
    pid = np.array([0, 0, 1], np.int64)
    with pytest.raises(P.SCCSError) as ei:
        P.sccs_create(3, pid, np.array([1, 0, 1], np.int32), np.ones(3), 1, np.array([0, 2], np.int64),
                      np.array([1, 1], np.int32))
    assert ei.value.code == -9


def test_edge_no_columns_and_max_cycles_zero(P):
    d, _ = tiny_fit_config()
    orc = oracle.Problem.from_data(d)
    with gpu_model(P, d) as m:
        m.set_prior("normal", 1.0)
        r = m.fit(max_cycles=0)
        assert r["cycles"] == 0 and r["rc"] == 1
        assert rel(r["logpost"], orc.logpost(np.zeros(d.J), "normal", 1.0)) <= 1e-12
    d0 = from_dense(d.patient_id, d.y, d.L, np.zeros((d.K, 0)))
    with gpu_model(P, d0) as m:
        r = m.fit(max_cycles=3, tol=-1.0)
        assert r["cycles"] == 3
        assert rel(r["logpost"], oracle.Problem.from_data(d0).loglik(np.zeros(0))) <= 1e-12


# ------------------------------------------------------------------ failure detection

def test_bounded_wait_times_out_and_handle_recovers(P):
    """One CTA fewer than the all-reduce counts: every wait must run out (~0.2 s), report
    SCCS_E_TIMEOUT, and leave a usable handle."""
    d, fit = tiny_fit_config()
    ref = oracle.Problem.from_data(d).fit(prior="normal", variance=1.0, fixed_cycles=2)
    with gpu_model(P, d) as m:
        rc = P.sccs_check_wait_timeout(m.handle, 200.0)
        assert rc == -6
        m.set_prior("normal", 1.0)
        r = m.fit(tol=-1.0, max_cycles=2)
    np.testing.assert_allclose(r["beta"], ref["beta"], atol=1e-11)


# ------------------------------------------------------------------ FP32 mode and FP64 polish

def _converged_oracle(d, prior, var, cycles=60):
    """The MAP to machine precision: a fixed, large number of cycles (a stop on |dP| resolves
    beta only to about sqrt(dP / curvature))."""
    return oracle.Problem.from_data(d).fit(prior=prior, variance=var, fixed_cycles=cycles)


@pytest.mark.parametrize("prior,var", [("normal", 0.1), ("laplace", 0.05)])
def test_fp32_phase_error_against_fp64_oracle(P, prior, var):
    """FP32 E, compensated per-subject sums and exact cross-subject sums: the FP32 fit lands
    within FP32 resolution of the FP64 MAP (the error is stated, and bounded here)."""
    d, _ = mid_fit_config(scale=0.02)
    ref = _converged_oracle(d, prior, var)
    with gpu_model(P, d) as m:
        m.set_prior(prior, var)
        r32 = m.fit(precision="fp32", tol_mode="rel_logpost", tol=1e-7, max_cycles=200)
    err = float(np.abs(r32["beta"] - ref["beta"]).max())
    print(f"FP32-only max |beta - beta_oracle| = {err:.3e} ({prior}, {r32['cycles']} cycles)")
    assert r32["fp32_cycles"] == r32["cycles"] > 0
    assert err <= 2e-4


@pytest.mark.parametrize("prior,var", [("normal", 0.1), ("laplace", 0.05)])
def test_fp32_polish_meets_fp64_bar(P, prior, var):
    """FP32 phase to a relative change of 1e-6, then FP64 cycles to convergence: the result
    meets the FP64 bar against the oracle's MAP (beta <= 1e-8, P <= 1e-10)."""
    d, _ = mid_fit_config(scale=0.02)
    ref = _converged_oracle(d, prior, var)
    with gpu_model(P, d) as m:
        m.set_prior(prior, var)
        r = m.fit(precision="fp32_polish", tol=-1.0, max_cycles=40)
    err = float(np.abs(r["beta"] - ref["beta"]).max())
    print(f"FP32+polish max |beta - beta_oracle| = {err:.3e} ({prior}, {r['fp32_cycles']} FP32 + "
          f"{r['cycles'] - r['fp32_cycles']} FP64 cycles)")
    assert r["fp32_cycles"] > 0 and r["cycles"] > r["fp32_cycles"]
    assert err <= 1e-8
    assert rel(r["logpost"], ref["logpost"]) <= 1e-10
    if prior == "laplace":
        assert np.array_equal(r["beta"] == 0, ref["beta"] == 0)


def test_fp32_grad_path_and_tiny_config(P):
    """The tiny workload in FP32+polish (every slice staged) and a config with slices too big to
    stage (3 shards), against the oracle's converged fit."""
    d, fit = tiny_fit_config()
    ref = _converged_oracle(d, "normal", 1.0)
    with gpu_model(P, d) as m:
        m.set_prior("normal", 1.0)
        r = m.fit(precision="fp32_polish", tol=-1.0, max_cycles=40)
    assert float(np.abs(r["beta"] - ref["beta"]).max()) <= 1e-8
    d2 = make_dataset(n_patients=60000, eras=("geometric", 8), J=10, columns=("density_range", 0.01, 0.2),
                      n_true=4, beta_sd=0.5, seed=31)
    ref2 = _converged_oracle(d2, "normal", 0.3)
    with gpu_model(P, d2, num_shards=3) as m:
        m.set_prior("normal", 0.3)
        r2 = m.fit(precision="fp32_polish", tol=-1.0, max_cycles=40)
        r32 = m.fit(precision="fp32", tol_mode="rel_logpost", tol=1e-7, max_cycles=200)
    assert float(np.abs(r2["beta"] - ref2["beta"]).max()) <= 1e-8
    assert float(np.abs(r32["beta"] - ref2["beta"]).max()) <= 2e-4


@pytest.mark.parametrize("prior,var", [("normal", 0.3), ("laplace", 0.1)])
def test_narrow_columns_match_wide_path_and_oracle(P, prior, var):
    """Columns run whole on one CTA (block-level sums) against the same fit with every column
    on all CTAs, and against the oracle: a mix of narrow and wide columns, narrow runs at the
    start and end of the cycle."""
    sizes = np.array([5, 3000, 40, 7, 12000, 900, 2, 60, 25000, 15, 300, 8, 1])
    d = make_dataset(n_patients=30000, eras=("geometric", 8), J=sizes.size, columns=("sizes", sizes),
                     n_true=4, beta_sd=0.5, seed=21)
    orc = oracle.Problem.from_data(d)
    ref = orc.fit(prior=prior, variance=var, fixed_cycles=4)
    out = {}
    for thr, gmax in ((-1, 0), (1000, 1), (1000, 0), (0, 0)):
        with gpu_model(P, d, num_shards=16, narrow_max_nnz=thr, narrow_group_max=gmax) as m:
            info = m.info
            m.set_prior(prior, var)
            out[thr if gmax == 0 else (thr, gmax)] = (m.fit(tol=-1.0, max_cycles=4, history=True),
                                                      info["narrow_columns"])
    assert out[-1][1] == 0 and 0 < out[1000][1] <= out[0][1] <= sizes.size
    for thr in (-1, 1000, 0, (1000, 1)):
        r = out[thr][0]
        np.testing.assert_allclose(r["beta"], ref["beta"], atol=1e-11, rtol=0)
        np.testing.assert_allclose(r["history"], ref["history"], rtol=1e-12)
        assert r["nonzero_steps"] == out[-1][0]["nonzero_steps"]


@pytest.mark.parametrize("prior,var", [("normal", 0.2), ("laplace", 0.05)])
def test_many_narrow_runs_between_wide_columns(P, prior, var):
    """400 columns: wide columns over a fifth of the subjects alternate with short runs of tiny
    columns, so most runs start on subjects the wide column before them has just changed (the
    run's first gather is speculative and must re-read exactly those).  Six fixed cycles of the
    narrow path, the all-wide path and the oracle agree to rounding."""
    rng = np.random.default_rng(77)
    sizes = []
    while len(sizes) < 400:
        sizes.append(int(rng.integers(2000, 6000)))                 # wide
        sizes.extend(int(x) for x in rng.integers(1, 80, size=int(rng.integers(1, 5))))   # a run
    sizes = np.array(sizes[:400])
    d = make_dataset(n_patients=20000, eras=("geometric", 6), J=sizes.size, columns=("sizes", sizes),
                     n_true=10, beta_sd=0.4, seed=78)
    orc = oracle.Problem.from_data(d)
    ref = orc.fit(prior=prior, variance=var, fixed_cycles=6)
    res = {}
    for thr in (0, -1):
        with gpu_model(P, d, num_shards=16, narrow_max_nnz=thr) as m:
            if thr == 0:
                assert m.info["narrow_columns"] > 150
            m.set_prior(prior, var)
            res[thr] = m.fit(tol=-1.0, max_cycles=6, history=True)
    for thr in (0, -1):
        np.testing.assert_allclose(res[thr]["beta"], ref["beta"], atol=1e-11, rtol=0)
        np.testing.assert_allclose(res[thr]["history"], ref["history"], rtol=1e-12)
    np.testing.assert_allclose(res[0]["beta"], res[-1]["beta"], atol=1e-12, rtol=0)
    assert res[0]["nonzero_steps"] == res[-1]["nonzero_steps"]


@pytest.mark.parametrize("shards", [2, 5])
def test_unstaged_slices_pipelined_gather(P, shards):
    """Columns far larger than a staged slice on few shards: phase A walks dozens of 32-segment
    groups per warp from global memory, the next group's row indices copied ahead into shared
    memory; segments up to 30 rows long also take the unstaged later diagonals.  Three fixed
    cycles against the oracle."""
    sizes = np.array([300000, 150000, 60000, 9000, 500, 20])
    d = make_dataset(n_patients=40000, eras=("uniform", 1, 30), J=sizes.size, columns=("sizes", sizes),
                     n_true=3, beta_sd=0.3, seed=95)
    orc = oracle.Problem.from_data(d)
    ref = orc.fit(prior="normal", variance=0.5, fixed_cycles=3)
    with gpu_model(P, d, num_shards=shards) as m:
        m.set_prior("normal", 0.5)
        r = m.fit(tol=-1.0, max_cycles=3, history=True)
    np.testing.assert_allclose(r["beta"], ref["beta"], atol=1e-11, rtol=0)
    np.testing.assert_allclose(r["history"], ref["history"], rtol=1e-12)


def test_all_columns_narrow_and_converged(P):
    d, fit = tiny_fit_config()
    orc = oracle.Problem.from_data(d)
    with gpu_model(P, d, num_shards=8, narrow_max_nnz=100000) as m:
        assert m.info["narrow_columns"] == d.J
        m.set_prior(fit["prior"], fit["variance"])
        r = m.fit(tol_mode="rel_logpost", tol=1e-15, max_cycles=200)
    compare_converged(r, orc, fit["prior"], fit["variance"], "rel_logpost", 1e-15)


def test_step_exponential_against_cuda_exp(P):
    """The table-driven e^x of the coordinate step against CUDA's exp and the host's: within an
    ulp of the host's everywhere (steps are small; the tails past |x| = 700 go to exp itself)."""
    rng = np.random.default_rng(3)
    small = 2.0 ** -10
    x = np.concatenate([rng.normal(0, 0.05, 200000), rng.uniform(-30, 30, 200000), rng.uniform(-699, 699, 50000),
                        rng.uniform(-small, small, 100000), rng.normal(0, 1e-7, 20000),
                        np.nextafter(small, 0) * np.array([1, -1]), small * np.array([1, -1]),
                        np.nextafter(small, 1) * np.array([1, -1]),
                        np.array([0.0, -0.0, 1e-300, -1e-300, 5e-17, -5e-17, 1.0, -1.0, 0.5 * np.log(2),
                                  np.log(2) / 64, -np.log(2) / 64, 699.9, -699.9, 700.0, -700.0, 709.0,
                                  -745.0, np.inf, -np.inf, np.nan])])
    ours, ref = P.sccs.sccs_selftest_exp(x)
    fin = np.isfinite(ref) & (ref > 0)
    ulp = np.abs(ours[fin] - ref[fin]) / np.spacing(ref[fin])
    with np.errstate(over="ignore"):
        host = np.exp(x[fin])
    ulp_host = np.abs(ours[fin] - host) / np.spacing(host)
    assert ulp.max() <= 2.0, ulp.max()          # two approximations within 1 ulp each
    assert ulp_host.max() <= 1.0, ulp_host.max()
    assert np.mean(ulp == 0) > 0.5
    assert ours[x == 0.0].tolist() == [1.0, 1.0]
    assert np.isnan(ours[-1]) and ours[-2] == 0.0 and np.isinf(ours[-3])


def test_step_quotient_against_ieee_division(P):
    """The coordinate path's quotient (FP32 reciprocal seed, Newton-Raphson refinement) against
    CUDA's IEEE division: within an ulp everywhere, the same bits nearly always, and the IEEE
    result itself for zeros, infinities, NaNs and magnitudes outside the seed's range."""
    rng = np.random.default_rng(11)
    n = 400000
    D = 10.0 ** rng.uniform(-6, 12, n)                    # W = num / D with 0 < num <= D
    num = D * rng.uniform(0, 1, n)
    g = rng.normal(0, 1e4, n)                               # Newton steps g / q
    q = 10.0 ** rng.uniform(-8, 8, n)
    specials_a = np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, np.nan, 1.0, 1.0, 1e-310, 1e300, 2.0 ** -901,
                           2.0 ** -900, 3.0, 5e-324, 1.0])
    specials_b = np.array([3.0, 3.0, 0.0, -0.0, 2.0, 2.0, 2.0, np.inf, np.nan, 3.0, 1e-10, 1.0, 1.0, 2.0 ** 121,
                           1.0, 2.0 ** -121])
    a = np.concatenate([num, g, specials_a])
    b = np.concatenate([D, q, specials_b])
    ours, ref = P.sccs.sccs_selftest_div(a, b)
    fin = np.isfinite(ref)
    assert np.array_equal(np.isnan(ours), np.isnan(ref))
    assert np.array_equal(ours[~fin & ~np.isnan(ref)], ref[~fin & ~np.isnan(ref)])
    nz = fin & (ref != 0)
    ulp = np.abs(ours[nz] - ref[nz]) / np.spacing(np.abs(ref[nz]))
    assert ulp.max() <= 1.0, ulp.max()
    assert np.mean(ours[fin] == ref[fin]) > 0.999
    k = len(specials_a)
    sa, so = ref[-k:], ours[-k:]
    same = (sa == so) | (np.isnan(sa) & np.isnan(so))
    assert same.all(), (sa, so)
    assert np.array_equal(np.signbit(so[:2]), np.signbit(sa[:2]))   # signed zeros kept


def _genkin_stat(X, b_now, b_prev):
    xb, xp = X @ b_now, X @ b_prev
    return np.abs(xb - xp).sum() / (1.0 + np.abs(xb).sum())


@pytest.mark.parametrize("tol", [5e-4, 1e-9])
def test_genkin_xbeta_rule_against_oracle(P, tol):
    """Genkin's relative change of X beta over a cycle (the paper's Section 2.2 criterion, tol
    0.0005 there): the GPU stops at the first cycle whose statistic, computed from the oracle's
    own trajectory with a dense X, is below tol; its beta is the oracle's at that cycle."""
    from sccs_testlib import to_dense
    d, fit = tiny_fit_config()
    orc = oracle.Problem.from_data(d)
    X = to_dense(d)
    with gpu_model(P, d) as m:
        m.set_prior("normal", 1.0)
        r = m.fit(tol_mode="genkin_xbeta", tol=tol, max_cycles=500)
        r32 = m.fit(tol_mode="genkin_xbeta", tol=tol, max_cycles=500, precision="fp32_polish")
        with pytest.raises(P.SCCSError) as ei:
            m.fit(tol_mode="genkin_xbeta", tol=tol, precision="fp32")
        assert ei.value.code == P.sccs.E_UNSUPPORTED
    c = r["cycles"]
    assert r["rc"] == 0 and c >= 1 and r32["rc"] == 0
    same = orc.fit(prior="normal", variance=1.0, fixed_cycles=c)
    prev = orc.fit(prior="normal", variance=1.0, fixed_cycles=c - 1)
    np.testing.assert_allclose(r["beta"], same["beta"], atol=1e-11, rtol=0)
    assert _genkin_stat(X, same["beta"], prev["beta"]) < tol * (1 + 1e-6)
    if c > 1:
        pprev = orc.fit(prior="normal", variance=1.0, fixed_cycles=c - 2)
        assert _genkin_stat(X, prev["beta"], pprev["beta"]) >= tol * (1 - 1e-6)
    ocycles = orc.fit(prior="normal", variance=1.0, tol_mode="genkin_xbeta", tol=tol, max_cycles=500)["cycles"]
    assert ocycles == c


@pytest.mark.fullsize
def test_paper_scale_sampled_against_oracle(P):
    """The paper-scale workload at full size (4M subjects, 5,000 drugs, ~1e9 nonzeros, Laplace) in
    FP32 + FP64 polish, checked on sampled outputs the oracle computes straight from the input
    arrays: L at the fitted beta, g_j and h_j of sampled columns (the largest, the smallest, the
    largest effects, random ones), and the Laplace optimality conditions with the oracle's g_j."""
    from synth import paper_scale_config
    d, fit = paper_scale_config()
    with gpu_model(P, d) as m:
        m.set_prior(fit["prior"], fit["variance"])
        r = m.fit(precision="fp32_polish", tol_mode="rel_logpost", tol=1e-15, max_cycles=60)
        beta = r["beta"]
        nnz = np.diff(d.col_ptr)
        rng = np.random.default_rng(0)
        cols = sorted({0, 1, int(np.argmax(nnz)), int(np.argmin(nnz)), *map(int, np.argsort(-np.abs(beta))[:3]),
                       *map(int, rng.choice(d.J, 5, replace=False))})
        gh = np.array([m.grad_hess(j, beta) for j in cols])
        ll_gpu = m.logpost(beta)[1]
    ll, g, h = oracle.raw_eval(d, beta, cols)
    assert rel(ll_gpu, ll) <= 1e-12
    scale = np.maximum(1.0, np.abs(h))
    np.testing.assert_array_less(np.abs(gh[:, 0] - g), 1e-9 * scale)
    np.testing.assert_array_less(np.abs(gh[:, 1] - h), 1e-9 * scale)
    lam = np.sqrt(2.0 / fit["variance"])
    b = beta[cols]
    nzs = b != 0
    np.testing.assert_array_less(np.abs(g[nzs] - lam * np.sign(b[nzs])), 1e-6 * scale[nzs])
    np.testing.assert_array_less(np.abs(g[~nzs]), lam + 1e-6 * scale[~nzs])
    assert nzs.sum() >= 3


def test_narrow_groups_of_independent_columns(P):
    """Many small narrow columns over many subjects: most neighbours touch disjoint subjects and
    share a group; the grouped fit equals the one-at-a-time narrow fit and the oracle."""
    d = make_dataset(n_patients=200000, eras=("geometric", 5), J=60, columns=("sizes", np.full(60, 40)),
                     n_true=6, beta_sd=0.5, seed=33)
    orc = oracle.Problem.from_data(d)
    ref = orc.fit(prior="normal", variance=0.4, fixed_cycles=3)
    res = []
    for gmax in (1, 0, 3):
        with gpu_model(P, d, num_shards=32, narrow_group_max=gmax) as m:
            assert m.info["narrow_columns"] == d.J
            m.set_prior("normal", 0.4)
            res.append(m.fit(tol=-1.0, max_cycles=3, history=True))
    for r in res:
        np.testing.assert_allclose(r["beta"], ref["beta"], atol=1e-11, rtol=0)
        np.testing.assert_allclose(r["history"], ref["history"], rtol=1e-12)
        assert r["nonzero_steps"] == res[0]["nonzero_steps"]


def test_long_fit_stays_on_the_oracle_trajectory(P):
    """The 1,000-cycle default cap run in full (tol < 0), long past convergence: E is updated
    multiplicatively (E_k <- E_k e^{db}) and rebuilt from beta every 64 cycles, the oracle
    recomputes l_k exp(Xb_k) at every update; after 1,000 cycles beta still agrees to 1e-10 and P
    to 1e-12.  The FP32 mode (rebuilt every 16 cycles) stays within its own bar."""
    d, _ = tiny_fit_config()
    orc = oracle.Problem.from_data(d)
    ref = orc.fit(prior="normal", variance=1.0, fixed_cycles=1000)
    with gpu_model(P, d) as m:
        m.set_prior("normal", 1.0)
        r = m.fit(tol=-1.0, max_cycles=1000)
        r32 = m.fit(tol=-1.0, max_cycles=1000, precision="fp32")
    assert r["cycles"] == 1000
    np.testing.assert_allclose(r["beta"], ref["beta"], atol=1e-10, rtol=0)
    assert rel(r["logpost"], ref["logpost"]) <= 1e-12
    assert np.abs(r32["beta"] - ref["beta"]).max() <= 2e-4
