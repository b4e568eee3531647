/*
 * sccs_oracle.c -- serial FP64 CPU oracle for the Bayesian self-controlled case series
 * (BSCCS) MAP fit by cyclic coordinate descent (Suchard et al., arXiv 1208.0945).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
 * baseline call this code.  The CUDA library shares nothing with it: not a header, not a
 * helper, not a table.  It is deliberately plain and slow: one thread, FP64 throughout,
 * every sum taken in ascending row / subject / column order, no blocking or fusion.
 *
 * What it computes (paper notation; "Eq." numbers count the paper's displayed equations):
 *   Eq. 1  per-subject conditional likelihood  prod_k (e^{x_ik'b} / sum_k' l_ik' e^{x_ik'b})^{y_ik}
 *   Eq. 2  L(b) = sum_i [ sum_k y_ik x_ik'b - n_i log sum_k l_ik e^{x_ik'b} ]
 *   Eq. 3  b_j ~ Normal(0, s2) or Laplace(0, s2), s2 the variance
 *   Eq. 4  Newton step  db_j = -(g_j + d log p) / (h_j + d2 log p)
 *   Eq. 7  g_j = Y'X_j - N'W,   Eq. 8  W = M[L x exp(Xb) x X_j] / M[L x exp(Xb)]
 *   Eq. 9  h_j = -N'[W x (1 - W)]
 *   Algorithm 1 (Section 2.2): b = 0, Xb = 0, L x exp(Xb) = L, M[..] = M L; cycle over
 *   j = 1..J; after each nonzero db_j update Xb, L x exp(Xb) and M[L x exp(Xb)]; repeat to
 *   convergence; report b_MAP and P(b_MAP).
 *   Section 2.3 steps 1-4: the updates touch only the rows of X_j (sparse updates).
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   R1 trust region (Genkin et al. 2007, cited in Section 2.2): db = clamp(dv, -T_j, T_j),
 *      T_j <- max(2|db|, T_j / 2), T_j = 1 initially; dv is the exact-Hessian Newton step.
 *   R2 Laplace(0, s2) with s2 the variance: lambda = sqrt(2 / s2).  Soft threshold: at b_j = 0
 *      try (g - lambda)/q > 0, else (g + lambda)/q < 0, else 0; at b_j != 0 with sign s take
 *      (g - lambda s)/q and stop at 0 instead of crossing it.
 *   R3 log-posterior drops every constant: P = L(b) - sum b^2 / (2 s2)  or  L(b) - lambda sum|b|.
 *   R4 convergence: |dP| < tol (abs), |dP| / max(1,|P|) < tol (rel), or Genkin's
 *      sum_k |dXb_k| / (1 + sum_k |Xb_k|) < tol, checked once per full cycle.
 *   R5 q = -h = 0: Normal prior still gives a finite step; Laplace with |g| <= lambda gives
 *      db = -b_j; otherwise the coordinate is unbounded and takes the trust bound in the
 *      direction of the penalised gradient (a warning bit is raised); no prior: same.
 *   R6 "if db_j != 0" is an exact-zero test.
 *   R7 the denominators M[L x exp(Xb)] are recomputed from L x exp(Xb) at the end of every
 *      cycle (the incremental update accumulates rounding otherwise).
 *   R8 subjects with n_i = 0 contribute nothing (Section 2.1) and are removed up front.
 *   R9 subject weights (Section 2.5): a non-negative integer w_i per input subject stands for
 *      subject i appearing w_i times.  The bootstrap's resample with replacement gives the
 *      multiplicities; a cross-validation fit on the other folds gives w_i = 1 outside the
 *      held-out fold and 0 inside it; the predictive log-likelihood of the held-out fold is
 *      Eq. 2 summed over that fold's subjects, i.e. weights 1 on the fold and 0 elsewhere.
 *      Weighted, Eq. 2 reads  L_w(b) = sum_i w_i [ sum_k y_ik x_ik'b - n_i log sum_k l_ik e^{x_ik'b} ],
 *      so Y'X_j becomes sum_k w_i(k) y_k x_kj and n_i becomes w_i n_i in Eqs. 7-9.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_NOT_CONVERGED 1
#define ORC_E_INVAL (-1)
#define ORC_E_UNSORTED (-2)
#define ORC_E_NOMEM (-4)
#define ORC_E_NUMERIC (-7)
#define ORC_E_DUPLICATE (-9)

#define ORC_PRIOR_NONE 0
#define ORC_PRIOR_NORMAL 1
#define ORC_PRIOR_LAPLACE 2

#define ORC_TOL_ABS_LOGPOST 0
#define ORC_TOL_REL_LOGPOST 1
#define ORC_TOL_GENKIN_XBETA 2

typedef struct {
    int64_t K;        /* rows kept (eras of subjects with n_i >= 1) */
    int64_t N;        /* subjects kept */
    int32_t J;        /* drug columns */
    int64_t nnz;      /* nonzeros kept */
    int64_t *pat_ptr; /* N+1: rows of subject i are pat_ptr[i] .. pat_ptr[i+1]-1 (the M of Eq. 5) */
    int64_t *row_pat; /* K: subject of each row */
    int64_t *y;       /* K: events y_k */
    double *L;        /* K: offsets l_k */
    int64_t *n;       /* N: n_i = sum_k y_ik */
    int64_t *col_ptr; /* J+1 */
    int64_t *rows;    /* nnz: rows of each column, ascending */
    int64_t *ytx;     /* J: Y'X_j (Eq. 7, first term) */
    int64_t *sub_in;  /* N: input subject index of each kept subject (R9 weights are per input subject) */
    int64_t n_in;     /* input subjects */
    int64_t dropped_patients, dropped_rows;
} oracle_problem;

static void *xcalloc(size_t n, size_t sz) { return calloc(n ? n : 1, sz ? sz : 1); }

void oracle_free(oracle_problem *p) {
    if (!p) return;
    free(p->pat_ptr); free(p->row_pat); free(p->y); free(p->L); free(p->n);
    free(p->col_ptr); free(p->rows); free(p->ytx); free(p->sub_in);
    free(p);
}

static int cmp_i64(const void *a, const void *b) {
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* Build the canonical problem: subjects with n_i = 0 removed (R8), rows renumbered,
 * column rows sorted ascending, duplicates rejected. */
oracle_problem *oracle_create(int64_t K, const int64_t *patient_id, const int32_t *y,
                              const double *L, int32_t J, const int64_t *col_ptr,
                              const int32_t *row_idx, int *err) {
    *err = ORC_OK;
    if (K < 0 || J < 0) { *err = ORC_E_INVAL; return NULL; }
    for (int64_t k = 1; k < K; ++k)
        if (patient_id[k] < patient_id[k - 1]) { *err = ORC_E_UNSORTED; return NULL; }
    for (int64_t k = 0; k < K; ++k)
        if (y[k] < 0 || !(L[k] > 0.0) || !isfinite(L[k])) { *err = ORC_E_INVAL; return NULL; }
    if (col_ptr[0] != 0) { *err = ORC_E_INVAL; return NULL; }
    for (int32_t j = 0; j < J; ++j)
        if (col_ptr[j + 1] < col_ptr[j]) { *err = ORC_E_INVAL; return NULL; }
    int64_t nnz_in = col_ptr[J];
    for (int64_t e = 0; e < nnz_in; ++e)
        if (row_idx[e] < 0 || (int64_t)row_idx[e] >= K) { *err = ORC_E_INVAL; return NULL; }

    oracle_problem *p = (oracle_problem *)xcalloc(1, sizeof(oracle_problem));
    if (!p) { *err = ORC_E_NOMEM; return NULL; }

    /* events per input subject (runs of equal patient_id) */
    int64_t nsub = 0;
    for (int64_t k = 0; k < K; ++k)
        if (k == 0 || patient_id[k] != patient_id[k - 1]) nsub++;
    int64_t *sub_start = (int64_t *)xcalloc((size_t)nsub + 1, sizeof(int64_t));
    int64_t *sub_n = (int64_t *)xcalloc((size_t)nsub, sizeof(int64_t));
    int64_t *newrow = (int64_t *)xcalloc((size_t)K, sizeof(int64_t));
    if (!sub_start || !sub_n || !newrow) { free(sub_start); free(sub_n); free(newrow); oracle_free(p); *err = ORC_E_NOMEM; return NULL; }
    int64_t s = -1;
    for (int64_t k = 0; k < K; ++k) {
        if (k == 0 || patient_id[k] != patient_id[k - 1]) { s++; sub_start[s] = k; }
        sub_n[s] += y[k];
    }
    sub_start[nsub] = K;

    int64_t Nk = 0, Kk = 0;
    for (int64_t i = 0; i < nsub; ++i)
        if (sub_n[i] > 0) { Nk++; Kk += sub_start[i + 1] - sub_start[i]; }
    p->N = Nk; p->K = Kk; p->J = J;
    p->dropped_patients = nsub - Nk; p->dropped_rows = K - Kk;
    p->pat_ptr = (int64_t *)xcalloc((size_t)Nk + 1, sizeof(int64_t));
    p->row_pat = (int64_t *)xcalloc((size_t)Kk, sizeof(int64_t));
    p->y = (int64_t *)xcalloc((size_t)Kk, sizeof(int64_t));
    p->L = (double *)xcalloc((size_t)Kk, sizeof(double));
    p->n = (int64_t *)xcalloc((size_t)Nk, sizeof(int64_t));
    p->col_ptr = (int64_t *)xcalloc((size_t)J + 1, sizeof(int64_t));
    p->ytx = (int64_t *)xcalloc((size_t)J, sizeof(int64_t));
    p->sub_in = (int64_t *)xcalloc((size_t)Nk, sizeof(int64_t));
    p->n_in = nsub;
    if (!p->pat_ptr || !p->row_pat || !p->y || !p->L || !p->n || !p->col_ptr || !p->ytx || !p->sub_in) {
        free(sub_start); free(sub_n); free(newrow); oracle_free(p); *err = ORC_E_NOMEM; return NULL;
    }
    int64_t i2 = 0, k2 = 0;
    for (int64_t i = 0; i < nsub; ++i) {
        if (sub_n[i] == 0) {
            for (int64_t k = sub_start[i]; k < sub_start[i + 1]; ++k) newrow[k] = -1;
            continue;
        }
        p->pat_ptr[i2] = k2;
        p->n[i2] = sub_n[i];
        p->sub_in[i2] = i;
        for (int64_t k = sub_start[i]; k < sub_start[i + 1]; ++k) {
            newrow[k] = k2;
            p->row_pat[k2] = i2;
            p->y[k2] = y[k];
            p->L[k2] = L[k];
            k2++;
        }
        i2++;
    }
    p->pat_ptr[Nk] = Kk;
    free(sub_start); free(sub_n);

    /* columns: map rows, drop removed ones, sort, reject duplicates */
    int64_t cnt = 0;
    for (int64_t e = 0; e < nnz_in; ++e)
        if (newrow[row_idx[e]] >= 0) cnt++;
    p->rows = (int64_t *)xcalloc((size_t)cnt, sizeof(int64_t));
    if (!p->rows) { free(newrow); oracle_free(p); *err = ORC_E_NOMEM; return NULL; }
    int64_t w = 0;
    for (int32_t j = 0; j < J; ++j) {
        p->col_ptr[j] = w;
        int64_t a = w;
        for (int64_t e = col_ptr[j]; e < col_ptr[j + 1]; ++e) {
            int64_t r = newrow[row_idx[e]];
            if (r >= 0) p->rows[w++] = r;
        }
        qsort(p->rows + a, (size_t)(w - a), sizeof(int64_t), cmp_i64);
        for (int64_t e = a + 1; e < w; ++e)
            if (p->rows[e] == p->rows[e - 1]) { free(newrow); oracle_free(p); *err = ORC_E_DUPLICATE; return NULL; }
        int64_t t = 0;
        for (int64_t e = a; e < w; ++e) t += p->y[p->rows[e]];
        p->ytx[j] = t;
    }
    p->col_ptr[J] = w;
    p->nnz = w;
    free(newrow);
    return p;
}

void oracle_dims(const oracle_problem *p, int64_t *out6) {
    out6[0] = p->K; out6[1] = p->N; out6[2] = p->J; out6[3] = p->nnz;
    out6[4] = p->dropped_patients; out6[5] = p->dropped_rows;
}

int64_t oracle_subjects_in(const oracle_problem *p) { return p->n_in; }

/* R9: weight of kept subject i (1 without weights). */
static int64_t weight_of(const oracle_problem *p, const int64_t *w_in, int64_t i) {
    return w_in ? w_in[p->sub_in[i]] : 1;
}

/* R9: w_i n_i per kept subject and sum_k w_i(k) y_k x_kj per column, from their definitions. */
static void weighted_counts(const oracle_problem *p, const int64_t *w_in, int64_t *wn, int64_t *wytx) {
    for (int64_t i = 0; i < p->N; ++i) wn[i] = weight_of(p, w_in, i) * p->n[i];
    for (int32_t j = 0; j < p->J; ++j) {
        int64_t t = 0;
        for (int64_t e = p->col_ptr[j]; e < p->col_ptr[j + 1]; ++e) {
            int64_t k = p->rows[e];
            t += weight_of(p, w_in, p->row_pat[k]) * p->y[k];
        }
        wytx[j] = t;
    }
}

/* Xb from scratch: for each column j, add b_j to its rows (column order ascending). */
static void xbeta_from_scratch(const oracle_problem *p, const double *beta, double *xb) {
    for (int64_t k = 0; k < p->K; ++k) xb[k] = 0.0;
    for (int32_t j = 0; j < p->J; ++j) {
        if (beta[j] == 0.0) continue;
        for (int64_t e = p->col_ptr[j]; e < p->col_ptr[j + 1]; ++e) xb[p->rows[e]] += beta[j];
    }
}

/* Eq. 2, evaluated directly from its definition; with weights (R9) each subject's term is
 * counted w_i times (w_in: per input subject, NULL = all 1). */
double oracle_loglik_w(const oracle_problem *p, const double *beta, const int64_t *w_in) {
    double *xb = (double *)xcalloc((size_t)p->K, sizeof(double));
    if (!xb) return NAN;
    xbeta_from_scratch(p, beta, xb);
    double total = 0.0;
    for (int64_t i = 0; i < p->N; ++i) {
        double lin = 0.0, den = 0.0;
        for (int64_t k = p->pat_ptr[i]; k < p->pat_ptr[i + 1]; ++k) {
            lin += (double)p->y[k] * xb[k];
            den += p->L[k] * exp(xb[k]);
        }
        total += (double)weight_of(p, w_in, i) * (lin - (double)p->n[i] * log(den));
    }
    free(xb);
    return total;
}

double oracle_loglik(const oracle_problem *p, const double *beta) { return oracle_loglik_w(p, beta, NULL); }

/* log p(b) with every constant dropped (R3). */
static double log_prior(int prior, double var, const double *beta, int32_t J) {
    double s = 0.0;
    if (prior == ORC_PRIOR_NORMAL) {
        for (int32_t j = 0; j < J; ++j) s += beta[j] * beta[j];
        return -s / (2.0 * var);
    }
    if (prior == ORC_PRIOR_LAPLACE) {
        double lambda = sqrt(2.0 / var);
        for (int32_t j = 0; j < J; ++j) s += fabs(beta[j]);
        return -lambda * s;
    }
    return 0.0;
}

double oracle_logpost(const oracle_problem *p, const double *beta, int prior, double var) {
    return oracle_loglik(p, beta) + log_prior(prior, var, beta, p->J);
}

/* Eqs. 7-9 from scratch at beta: W_i = sum_{k in X_j, k in i} l_k e^{Xb_k} / sum_{k in i} l_k e^{Xb_k}. */
int oracle_grad_hess_w(const oracle_problem *p, const double *beta, int32_t j, const int64_t *w_in,
                       double *g, double *h) {
    if (j < 0 || j >= p->J) return ORC_E_INVAL;
    double *xb = (double *)xcalloc((size_t)p->K, sizeof(double));
    double *D = (double *)xcalloc((size_t)p->N, sizeof(double));
    double *num = (double *)xcalloc((size_t)p->N, sizeof(double));
    if (!xb || !D || !num) { free(xb); free(D); free(num); return ORC_E_NOMEM; }
    xbeta_from_scratch(p, beta, xb);
    for (int64_t k = 0; k < p->K; ++k) D[p->row_pat[k]] += p->L[k] * exp(xb[k]);
    for (int64_t e = p->col_ptr[j]; e < p->col_ptr[j + 1]; ++e) {
        int64_t k = p->rows[e];
        num[p->row_pat[k]] += p->L[k] * exp(xb[k]);
    }
    double nW = 0.0, nWW = 0.0;
    int64_t ytx = 0;
    for (int64_t e = p->col_ptr[j]; e < p->col_ptr[j + 1]; ++e)
        ytx += weight_of(p, w_in, p->row_pat[p->rows[e]]) * p->y[p->rows[e]];
    for (int64_t i = 0; i < p->N; ++i) {
        double Wi = num[i] / D[i];
        double ni = (double)(weight_of(p, w_in, i) * p->n[i]);
        nW += ni * Wi;
        nWW += ni * Wi * (1.0 - Wi);
    }
    *g = (double)ytx - nW;
    *h = -nWW;
    free(xb); free(D); free(num);
    return ORC_OK;
}

int oracle_grad_hess(const oracle_problem *p, const double *beta, int32_t j, double *g, double *h) {
    return oracle_grad_hess_w(p, beta, j, NULL, g, h);
}

/* The coordinate step of Eq. 4 under the prior (R2, R5) and the trust region (R1).
 * Returns db; updates *trust; sets *warn when the coordinate was unbounded. */
static double coordinate_step(double g, double h, double bj, int prior, double var,
                              double *trust, int *warn) {
    double q = -h; /* curvature of -L along e_j, >= 0 */
    double dv = 0.0;
    if (prior == ORC_PRIOR_NORMAL) {
        /* d log p = -b/s2, d2 log p = -1/s2 */
        dv = (g - bj / var) / (q + 1.0 / var);
    } else if (prior == ORC_PRIOR_LAPLACE) {
        double lambda = sqrt(2.0 / var);
        if (q > 0.0) {
            if (bj == 0.0) {
                double up = (g - lambda) / q, dn = (g + lambda) / q;
                if (up > 0.0) dv = up;
                else if (dn < 0.0) dv = dn;
                else dv = 0.0;
            } else {
                double s = bj > 0.0 ? 1.0 : -1.0;
                dv = (g - lambda * s) / q;
                double nb = bj + dv;
                double ns = nb > 0.0 ? 1.0 : (nb < 0.0 ? -1.0 : 0.0);
                if (ns != s) dv = -bj;
            }
        } else {
            if (bj == 0.0) {
                if (fabs(g) <= lambda) dv = 0.0;
                else { dv = (g > 0.0 ? 1.0 : -1.0) * (*trust); *warn = 1; }
            } else {
                double s = bj > 0.0 ? 1.0 : -1.0;
                if (fabs(g) <= lambda) dv = -bj;
                else {
                    double d = g - lambda * s;
                    dv = (d > 0.0 ? 1.0 : (d < 0.0 ? -1.0 : 0.0)) * (*trust);
                    double nb = bj + dv;
                    double ns = nb > 0.0 ? 1.0 : (nb < 0.0 ? -1.0 : 0.0);
                    if (ns != s) dv = -bj;
                    *warn = 1;
                }
            }
        }
    } else {
        if (q > 0.0) dv = g / q;
        else if (g != 0.0) { dv = (g > 0.0 ? 1.0 : -1.0) * (*trust); *warn = 1; }
        else dv = 0.0;
    }
    double db = dv;
    if (db > *trust) db = *trust;
    if (db < -*trust) db = -*trust;
    double t2 = 2.0 * fabs(db), th = 0.5 * (*trust);
    *trust = t2 > th ? t2 : th;
    return db;
}

/* Algorithm 1.  hist[0] = P(b0), hist[t] = P after cycle t (length max_cycles + 1).
 * tol < 0 runs exactly max_cycles cycles.  Returns ORC_OK, ORC_NOT_CONVERGED or an error. */
int oracle_fit_w(const oracle_problem *p, int prior, double var, int tol_mode, double tol,
                 int max_cycles, const double *beta0, const int64_t *w_in, double *beta_out, double *hist,
                 int *cycles_out, int64_t *nonzero_steps_out, int *warn_out) {
    if ((prior == ORC_PRIOR_NORMAL || prior == ORC_PRIOR_LAPLACE) && !(var > 0.0)) return ORC_E_INVAL;
    if (max_cycles < 0) return ORC_E_INVAL;
    const int64_t K = p->K, N = p->N;
    const int32_t J = p->J;
    double *beta = beta_out;
    double *xb = (double *)xcalloc((size_t)K, sizeof(double));
    double *xb_prev = (double *)xcalloc((size_t)K, sizeof(double));
    double *E = (double *)xcalloc((size_t)K, sizeof(double));
    double *D = (double *)xcalloc((size_t)N, sizeof(double));
    double *trust = (double *)xcalloc((size_t)J, sizeof(double));
    int64_t *wn = (int64_t *)xcalloc((size_t)N, sizeof(int64_t));    /* R9: w_i n_i */
    int64_t *wytx = (int64_t *)xcalloc((size_t)J, sizeof(int64_t));  /* R9: weighted Y'X_j */
    int64_t *wy = (int64_t *)xcalloc((size_t)K, sizeof(int64_t));    /* R9: w_i(k) y_k */
    if (!xb || !xb_prev || !E || !D || !trust || !wn || !wytx || !wy) {
        free(xb); free(xb_prev); free(E); free(D); free(trust); free(wn); free(wytx); free(wy);
        return ORC_E_NOMEM;
    }
    weighted_counts(p, w_in, wn, wytx);
    for (int64_t k = 0; k < K; ++k) wy[k] = weight_of(p, w_in, p->row_pat[k]) * p->y[k];
    for (int32_t j = 0; j < J; ++j) { beta[j] = beta0 ? beta0[j] : 0.0; trust[j] = 1.0; }

    /* Initialise: Xb, L x exp(Xb), M[L x exp(Xb)] (b = 0 gives Xb = 0, E = L, D = M L). */
    xbeta_from_scratch(p, beta, xb);
    for (int64_t k = 0; k < K; ++k) E[k] = p->L[k] * exp(xb[k]);
    for (int64_t i = 0; i < N; ++i) {
        double s = 0.0;
        for (int64_t k = p->pat_ptr[i]; k < p->pat_ptr[i + 1]; ++k) s += E[k];
        D[i] = s;
    }
    double ylin = 0.0, nlog = 0.0;
    for (int64_t k = 0; k < K; ++k) ylin += (double)wy[k] * xb[k];
    for (int64_t i = 0; i < N; ++i) nlog += (double)wn[i] * log(D[i]);
    double P_prev = ylin - nlog + log_prior(prior, var, beta, J);
    if (hist) hist[0] = P_prev;

    int status = ORC_NOT_CONVERGED, warn = 0, t = 0;
    int64_t nonzero_steps = 0;
    for (t = 1; t <= max_cycles; ++t) {
        if (tol_mode == ORC_TOL_GENKIN_XBETA) memcpy(xb_prev, xb, (size_t)K * sizeof(double));
        for (int32_t j = 0; j < J; ++j) {
            /* Eqs. 7-9 over the subjects X_j touches (W_i = 0 for the others). */
            double nW = 0.0, nWW = 0.0, num = 0.0;
            int64_t cur = -1;
            for (int64_t e = p->col_ptr[j]; e < p->col_ptr[j + 1]; ++e) {
                int64_t k = p->rows[e], i = p->row_pat[k];
                if (i != cur) {
                    if (cur >= 0) {
                        double Wi = num / D[cur];
                        nW += (double)wn[cur] * Wi;
                        nWW += (double)wn[cur] * Wi * (1.0 - Wi);
                    }
                    cur = i; num = 0.0;
                }
                num += E[k];
            }
            if (cur >= 0) {
                double Wi = num / D[cur];
                nW += (double)wn[cur] * Wi;
                nWW += (double)wn[cur] * Wi * (1.0 - Wi);
            }
            double g = (double)wytx[j] - nW, h = -nWW;
            double db = coordinate_step(g, h, beta[j], prior, var, &trust[j], &warn);
            if (!isfinite(db)) { status = ORC_E_NUMERIC; goto done; }
            if (db != 0.0) { /* R6 */
                nonzero_steps++;
                beta[j] += db;
                /* Section 2.3 steps 1-3, touching the rows of X_j only (Listing 3's update). */
                for (int64_t e = p->col_ptr[j]; e < p->col_ptr[j + 1]; ++e) {
                    int64_t k = p->rows[e];
                    xb[k] += db;
                    double En = p->L[k] * exp(xb[k]);
                    D[p->row_pat[k]] += En - E[k];
                    E[k] = En;
                }
            }
        }
        /* End of cycle: refresh the denominators (R7), evaluate P, test convergence (R4). */
        for (int64_t i = 0; i < N; ++i) {
            double s = 0.0;
            for (int64_t k = p->pat_ptr[i]; k < p->pat_ptr[i + 1]; ++k) s += E[k];
            D[i] = s;
        }
        ylin = 0.0; nlog = 0.0;
        for (int64_t k = 0; k < K; ++k) ylin += (double)wy[k] * xb[k];
        for (int64_t i = 0; i < N; ++i) nlog += (double)wn[i] * log(D[i]);
        double P = ylin - nlog + log_prior(prior, var, beta, J);
        if (!isfinite(P)) { status = ORC_E_NUMERIC; goto done; }
        if (hist) hist[t] = P;
        double conv;
        if (tol_mode == ORC_TOL_ABS_LOGPOST) conv = fabs(P - P_prev);
        else if (tol_mode == ORC_TOL_REL_LOGPOST) conv = fabs(P - P_prev) / (fabs(P) > 1.0 ? fabs(P) : 1.0);
        else {
            double dsum = 0.0, asum = 0.0;
            for (int64_t k = 0; k < K; ++k) { dsum += fabs(xb[k] - xb_prev[k]); asum += fabs(xb[k]); }
            conv = dsum / (1.0 + asum);
        }
        P_prev = P;
        if (tol >= 0.0 && conv < tol) { status = ORC_OK; break; }
    }
    if (t > max_cycles) t = max_cycles;
done:
    if (cycles_out) *cycles_out = t;
    if (nonzero_steps_out) *nonzero_steps_out = nonzero_steps;
    if (warn_out) *warn_out = warn;
    free(xb); free(xb_prev); free(E); free(D); free(trust); free(wn); free(wytx); free(wy);
    return status;
}

int oracle_fit(const oracle_problem *p, int prior, double var, int tol_mode, double tol,
               int max_cycles, const double *beta0, double *beta_out, double *hist,
               int *cycles_out, int64_t *nonzero_steps_out, int *warn_out) {
    return oracle_fit_w(p, prior, var, tol_mode, tol, max_cycles, beta0, NULL, beta_out, hist,
                        cycles_out, nonzero_steps_out, warn_out);
}

/* Eq. 2 and Eqs. 7-9 straight from the input arrays (no canonical copy: for sampled checks of
 * very large problems).  One pass builds Xb per row from scratch, one the denominators and n_i
 * per input subject (a run of equal patient_id; subjects with n_i = 0 contribute nothing, R8),
 * then L(b) and, for each requested column, g_j = Y'X_j - sum_i n_i W_ij and
 * h_j = -sum_i n_i W_ij (1 - W_ij).  Rows of a column may come in any order.  Returns ORC_OK,
 * ORC_E_INVAL or ORC_E_NOMEM. */
int oracle_raw_eval(int64_t K, const int64_t *patient_id, const int32_t *y, const double *L, int32_t J,
                    const int64_t *col_ptr, const int32_t *row_idx, const double *beta, int32_t ncols,
                    const int32_t *cols, double *loglik_out, double *g_out, double *h_out) {
    if (K < 0 || J < 0 || ncols < 0) return ORC_E_INVAL;
    for (int32_t c = 0; c < ncols; ++c)
        if (cols[c] < 0 || cols[c] >= J) return ORC_E_INVAL;
    double *xb = (double *)xcalloc((size_t)K, sizeof(double));
    int64_t *sub = (int64_t *)xcalloc((size_t)K, sizeof(int64_t));
    if (!xb || !sub) { free(xb); free(sub); return ORC_E_NOMEM; }
    for (int32_t j = 0; j < J; ++j) {
        if (beta[j] == 0.0) continue;
        for (int64_t e = col_ptr[j]; e < col_ptr[j + 1]; ++e) xb[row_idx[e]] += beta[j];
    }
    int64_t nsub = 0;
    for (int64_t k = 0; k < K; ++k) {
        if (k == 0 || patient_id[k] != patient_id[k - 1]) nsub++;
        sub[k] = nsub - 1;
    }
    double *D = (double *)xcalloc((size_t)nsub, sizeof(double));
    double *num = (double *)xcalloc((size_t)nsub, sizeof(double));
    int64_t *n = (int64_t *)xcalloc((size_t)nsub, sizeof(int64_t));
    if (!D || !num || !n) { free(xb); free(sub); free(D); free(num); free(n); return ORC_E_NOMEM; }
    double lin = 0.0;
    for (int64_t k = 0; k < K; ++k) {
        D[sub[k]] += L[k] * exp(xb[k]);
        n[sub[k]] += y[k];
        lin += (double)y[k] * xb[k];
    }
    double nlog = 0.0;
    for (int64_t i = 0; i < nsub; ++i)
        if (n[i] > 0) nlog += (double)n[i] * log(D[i]);
    if (loglik_out) *loglik_out = lin - nlog;
    for (int32_t c = 0; c < ncols; ++c) {
        const int32_t j = cols[c];
        int64_t ytx = 0;
        for (int64_t e = col_ptr[j]; e < col_ptr[j + 1]; ++e) {
            const int64_t k = row_idx[e];
            num[sub[k]] += L[k] * exp(xb[k]);
            if (n[sub[k]] > 0) ytx += y[k];
        }
        double nW = 0.0, nWW = 0.0;
        for (int64_t e = col_ptr[j]; e < col_ptr[j + 1]; ++e) {
            const int64_t i = sub[row_idx[e]];
            if (num[i] == 0.0) continue;      /* this subject's term was taken already */
            if (n[i] > 0) {
                const double Wi = num[i] / D[i];
                nW += (double)n[i] * Wi;
                nWW += (double)n[i] * Wi * (1.0 - Wi);
            }
            num[i] = 0.0;
        }
        g_out[c] = (double)ytx - nW;
        h_out[c] = -nWW;
    }
    free(xb); free(sub); free(D); free(num); free(n);
    return ORC_OK;
}
