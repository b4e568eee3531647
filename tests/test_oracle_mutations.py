"""The oracle's pins are sensitive: each plausible mistake planted in a copy of the oracle
source (a dropped term, a flipped sign, a wrong index, a wrong prior scale) makes at least
one pin fail.  Mistakes are planted only in a temporary CPU build of the oracle."""
import os
import shutil
import subprocess

import pytest

import oracle
import test_oracle_pins as pins
import test_oracle_weights as wpins

SRC = os.path.join(os.path.dirname(oracle.__file__), "sccs_oracle.c")

# (name, exact text in the oracle, replacement)
MUTATIONS = [
    ("hessian_sign_1_plus_w", "nWW += ni * Wi * (1.0 - Wi);", "nWW += ni * Wi * (1.0 + Wi);"),
    ("gradient_sign", "*g = (double)ytx - nW;", "*g = (double)ytx + nW;"),
    ("loglik_dropped_log_term", "(lin - (double)p->n[i] * log(den))", "(lin - log(den))"),
    ("laplace_scale", "double lambda = sqrt(2.0 / var);\n        if (q > 0.0)",
     "double lambda = sqrt(1.0 / var);\n        if (q > 0.0)"),
    ("normal_prior_curvature", "dv = (g - bj / var) / (q + 1.0 / var);", "dv = (g - bj / var) / (q + 2.0 / var);"),
    ("denominator_update_dropped_old", "D[p->row_pat[k]] += En - E[k];", "D[p->row_pat[k]] += En;"),
    ("off_by_one_subject", "if (cur >= 0) {\n                        double Wi = num / D[cur];",
     "if (cur >= 0) {\n                        double Wi = num / D[cur > 0 ? cur - 1 : 0];"),
    ("offset_ignored_in_update", "double En = p->L[k] * exp(xb[k]);", "double En = exp(xb[k]);"),
    # subject weights (Section 2.5)
    ("weights_ignored_in_ytx", "t += weight_of(p, w_in, p->row_pat[k]) * p->y[k];", "t += p->y[k];"),
    ("weights_ignored_in_n", "wn[i] = weight_of(p, w_in, i) * p->n[i];", "wn[i] = p->n[i];"),
    ("weights_ignored_in_loglik", "total += (double)weight_of(p, w_in, i) * (", "total += ("),
    ("weights_by_kept_subject", "return w_in ? w_in[p->sub_in[i]] : 1;", "return w_in ? w_in[i] : 1;"),
    # the evaluation straight from the input arrays
    ("raw_eval_unweighted_W", "nW += (double)n[i] * Wi;", "nW += Wi;"),
    ("raw_eval_counts_zero_event_rows", "if (n[sub[k]] > 0) ytx += y[k];", "ytx += y[k] + (n[sub[k]] == 0);"),
    # the Genkin trust region and convergence rule (Section 2.2)
    ("trust_update_factor", "double t2 = 2.0 * fabs(db), th = 0.5 * (*trust);",
     "double t2 = fabs(db), th = 0.5 * (*trust);"),
    ("trust_initial_radius", "beta[j] = beta0 ? beta0[j] : 0.0; trust[j] = 1.0;",
     "beta[j] = beta0 ? beta0[j] : 0.0; trust[j] = 2.0;"),
    ("genkin_drops_one_plus", "conv = dsum / (1.0 + asum);", "conv = dsum / asum;"),
    ("genkin_previous_cycle_not_saved",
     "if (tol_mode == ORC_TOL_GENKIN_XBETA) memcpy(xb_prev, xb, (size_t)K * sizeof(double));",
     "if (tol_mode == ORC_TOL_GENKIN_XBETA && t == 1) memcpy(xb_prev, xb, (size_t)K * sizeof(double));"),
    # q = 0 (R5): a nonzero Laplace coefficient with |g| <= lambda returns to 0
    ("laplace_q_zero_keeps_beta", "if (fabs(g) <= lambda) dv = -bj;", "if (fabs(g) <= lambda) dv = 0.0;"),
]

PIN_CASES = [
    (pins.test_loglik_equals_conditional_multinomial, dict(seed=0)),
    (pins.test_grad_hess_finite_differences, dict(seed=0)),
    (pins.test_grad_hess_against_dense_softmax_form, {}),
    (pins.test_golden_one_covariate_closed_forms, {}),
    (pins.test_one_covariate_general_minimiser, dict(seed=0)),
    (pins.test_ccd_matches_multivariate_newton, dict(seed=1, prior="normal")),
    (pins.test_laplace_kkt_certificate, dict(seed=1, var=0.2)),
    (wpins.test_weighted_fit_equals_replicated_dataset, dict(seed=0, prior="normal", var=0.5)),
    (wpins.test_fold_fit_and_heldout_loglik, dict(seed=0)),
    (pins.test_raw_eval_equals_canonical_oracle, dict(seed=0)),
    (pins.test_golden_trust_region_trajectory, {}),
    (pins.test_genkin_xbeta_stopping_rule, dict(seed=2)),
    (pins.test_column_covering_whole_subjects_q_zero, {}),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, name, old, new):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    mutated = tmp_path / "mut.c"
    mutated.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.run(oracle.compile_command(str(mutated), str(so)), check=True)
    lib = oracle.load_variant(str(so))
    failed = []
    saved = pins.ORACLE_LIB, wpins.ORACLE_LIB
    pins.ORACLE_LIB = wpins.ORACLE_LIB = lib
    try:
        for fn, kw in PIN_CASES:
            try:
                fn(**kw)
            except (AssertionError, oracle.OracleError):
                failed.append(fn.__name__)
    finally:
        pins.ORACLE_LIB, wpins.ORACLE_LIB = saved
    assert failed, f"planted mistake {name} passed every pin"


def test_unmutated_oracle_passes_the_same_pins():
    for fn, kw in PIN_CASES:
        fn(**kw)
