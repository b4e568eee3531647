// sccs_kernels.cu -- sm_103a kernels for the BSCCS cyclic-coordinate-descent MAP fit.
//
// One persistent cooperative launch runs a whole fit (Algorithm 1).  CTA s owns subject
// shard s: the eras (rows) and subjects in it, their L x exp(Xb) (E) and M[L x exp(Xb)] (D).
// Per coordinate j every CTA
//   A  gathers E at the nonzeros of its slice of X_j, sums them per subject (the numerator
//      M[L x exp(Xb) x X_j] of Eq. 8, restricted to the touched subjects), forms
//      W_i = num_i / D_i and the partial sums  sum n_i W_i  and  sum n_i W_i (1 - W_i)
//      (the fused transformation and reduction of Section 2.4, with W never stored);
//   -  joins one grid all-reduce of the two partials (fixed summation order, so all CTAs
//      hold bit-identical totals), then computes g_j, h_j (Eqs. 7, 9) and the step db_j
//      (Eq. 4 with the prior of Eq. 3 and a Genkin trust region) redundantly;
//   C  if db_j != 0, updates its own rows and subjects (Section 2.3 steps 1-3):
//      E_k <- E_k e^{db}  (= l_k exp(Xb_k + db), one exp per coordinate instead of one per
//      nonzero), and D_i <- D_i + (e^{db} - 1) num_i (= D_i + sum_k (E_k,new - E_k,old)).
// Because no CTA ever touches another shard's rows, phase C needs no grid barrier: the only
// cross-CTA traffic is the 16-byte partial per CTA per coordinate.  At the end of a cycle
// each CTA recomputes D from E on its subjects, and the log-posterior is all-reduced.
//
// Every wait is bounded by a deadline on %globaltimer; a CTA that gives up raises the abort
// flag and returns, and the others see the flag and return too.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "sccs_internal.h"

namespace sccs {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kUnroll = 4;       // diagonals of a warp's first group held in registers
constexpr int kMaxWarps = 32;

// status values written to FitOut
constexpr int kStOk = 0;
constexpr int kStNotConverged = 1;
constexpr int kStTimeout = -6;
constexpr int kStNumeric = -7;

__device__ __forceinline__ long long now_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ int ld_relaxed_i32(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// A non-negative double with its sign bit replaced by the phase bit.
__device__ __forceinline__ unsigned long long enc(double v, unsigned long long phase) {
    unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(fabs(v)));
    return (b & 0x7fffffffffffffffull) | (phase << 63);
}
__device__ __forceinline__ double dec(unsigned long long b) {
    return __longlong_as_double(static_cast<long long>(b & 0x7fffffffffffffffull));
}

// Grid all-reduce of two non-negative partials, run by one full warp of every CTA.
// Slot buffer (seq & 1) holds this round; the sign bit of each value equals the round's
// phase ((seq >> 1) & 1) ^ 1, which differs from what the buffer held two rounds earlier,
// so a reader can tell a fresh value from a stale one without any separate flag.  A CTA can
// not run two rounds ahead of a reader, because the round after next needs the reader's
// own contribution.  Totals are summed in the same order by every CTA (lane-strided, then a
// fixed tree read from lane 0), so all CTAs hold identical results.
__device__ bool grid_allreduce2(const DevLayout &d, unsigned long long seq, double a, double b,
                                double &A, double &B, long long timeout_ns) {
    const int lane = threadIdx.x & 31;
    const long long deadline = now_ns() + timeout_ns;
    const unsigned long long phase = ((seq >> 1) & 1ull) ^ 1ull;
    unsigned long long *buf = d.slots + (seq & 1ull) * 2ull * static_cast<unsigned long long>(d.S);
    if (lane == 0) {
        st_relaxed_u64(buf + 2 * blockIdx.x, enc(a, phase));
        st_relaxed_u64(buf + 2 * blockIdx.x + 1, enc(b, phase));
    }
    double sa, sb;
    for (int it = 0;; ++it) {
        bool ready = true;
        sa = 0.0;
        sb = 0.0;
        for (int s = lane; s < d.S; s += 32) {
            unsigned long long va = ld_relaxed_u64(buf + 2 * s);
            unsigned long long vb = ld_relaxed_u64(buf + 2 * s + 1);
            ready &= ((va >> 63) == phase) && ((vb >> 63) == phase);
            sa += dec(va);
            sb += dec(vb);
        }
        if (__all_sync(kFull, ready)) break;
        int give_up = 0;
        if (lane == 0 && (it & 15) == 15)
            give_up = (ld_relaxed_i32(d.abort_flag) != 0) || (now_ns() > deadline);
        if (__shfl_sync(kFull, give_up, 0)) {
            if (lane == 0) atomicExch(d.abort_flag, 1);
            return false;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sa += __shfl_down_sync(kFull, sa, o);
        sb += __shfl_down_sync(kFull, sb, o);
    }
    A = __shfl_sync(kFull, sa, 0);
    B = __shfl_sync(kFull, sb, 0);
    return true;
}

// Warp sum with a fixed association; the result is read from lane 0.
__device__ __forceinline__ double warp_sum_lane0(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
}

// Coordinate step: Newton step of Eq. 4 under the prior of Eq. 3, then the Genkin trust
// region.  q = -h >= 0.  Laplace: soft threshold at 0, and a step that would change the
// sign of a nonzero b stops at 0.  q = 0 with no finite minimiser takes the trust bound
// and raises warning bit 0.
__device__ double newton_step(double g, double h, double b, int prior, double var, double lambda,
                              double &trust, int &warn) {
    const double q = -h;
    double dv;
    if (prior == 1) {
        dv = (g - b / var) / (q + 1.0 / var);
    } else if (prior == 2) {
        if (q > 0.0) {
            if (b == 0.0) {
                const double up = (g - lambda) / q, dn = (g + lambda) / q;
                dv = up > 0.0 ? up : (dn < 0.0 ? dn : 0.0);
            } else {
                const double s = b > 0.0 ? 1.0 : -1.0;
                dv = (g - lambda * s) / q;
                const double nb = b + dv;
                const double ns = nb > 0.0 ? 1.0 : (nb < 0.0 ? -1.0 : 0.0);
                if (ns != s) dv = -b;
            }
        } else if (b == 0.0) {
            if (fabs(g) <= lambda) {
                dv = 0.0;
            } else {
                dv = (g > 0.0 ? 1.0 : -1.0) * trust;
                warn |= 1;
            }
        } else {
            const double s = b > 0.0 ? 1.0 : -1.0;
            if (fabs(g) <= lambda) {
                dv = -b;
            } else {
                const double dd = g - lambda * s;
                dv = (dd > 0.0 ? 1.0 : (dd < 0.0 ? -1.0 : 0.0)) * trust;
                const double nb = b + dv;
                const double ns = nb > 0.0 ? 1.0 : (nb < 0.0 ? -1.0 : 0.0);
                if (ns != s) dv = -b;
                warn |= 1;
            }
        }
    } else {
        if (q > 0.0) {
            dv = g / q;
        } else if (g != 0.0) {
            dv = (g > 0.0 ? 1.0 : -1.0) * trust;
            warn |= 1;
        } else {
            dv = 0.0;
        }
    }
    const double db = fmin(fmax(dv, -trust), trust);
    trust = fmax(2.0 * fabs(db), 0.5 * trust);
    return db;
}

// What a lane keeps between phases A and C for its warp's first group of the slice.
struct LaneCache {
    int32_t row[kUnroll];
    double e[kUnroll];
    int32_t pid;
    int32_t len;
    double Dv;
    double num;
    int64_t tail_base;   // rows[] index of diagonal kUnroll of the group
};

// Phase A for one group of 32 segments.  Adds this lane's n_i W_i and n_i W_i (1 - W_i)
// to G and H.  Keeps the lane's data in `lc` (first group of the warp) or in `stash`.
__device__ __forceinline__ void group_phase_a(const DevLayout &d, int64_t si, int64_t seg_end,
                                              int64_t base, double &G, double &H, LaneCache *lc,
                                              double *stash_slot) {
    const int lane = threadIdx.x & 31;
    const bool valid = si < seg_end;
    const int2 sg = valid ? d.segs[si] : make_int2(0, 0);
    const double Dv = valid ? d.D[sg.x] : 1.0;
    const int nv = valid ? d.nev[sg.x] : 0;
    const int maxlen = __shfl_sync(kFull, sg.y, 0);  // segments are sorted longest first
    double num = 0.0;
    int64_t b = base;
    int32_t rr[kUnroll];
    double ee[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
        const bool act = sg.y > u;
        const unsigned m = __ballot_sync(kFull, act);
        rr[u] = act ? d.rows[b + lane] : -1;
        b += __popc(m);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) ee[u] = rr[u] >= 0 ? d.E[rr[u]] : 0.0;
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) num += ee[u];
    const int64_t tail_base = b;
    for (int t = kUnroll; t < maxlen; t += kUnroll) {
        int32_t r2[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const bool act = sg.y > t + u;
            const unsigned m = __ballot_sync(kFull, act);
            r2[u] = act ? d.rows[b + lane] : -1;
            b += __popc(m);
        }
        double e2[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) e2[u] = r2[u] >= 0 ? d.E[r2[u]] : 0.0;
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) num += e2[u];
    }
    // W_i is a share of D_i; rounding in the incremental D can push it an ulp past 1.
    double w = valid ? num / Dv : 0.0;
    w = fmin(fmax(w, 0.0), 1.0);
    const double nw = static_cast<double>(nv) * w;
    G += nw;
    H += nw * (1.0 - w);
    if (lc) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            lc->row[u] = rr[u];
            lc->e[u] = ee[u];
        }
        lc->pid = valid ? sg.x : -1;
        lc->len = sg.y;
        lc->Dv = Dv;
        lc->num = num;
        lc->tail_base = tail_base;
    } else if (valid) {
        stash_slot[0] = num;
        stash_slot[1] = Dv;
    }
}

// Phase C for the tail diagonals (t >= from) of a group: E_k <- E_k * r.
__device__ __forceinline__ void group_tail_update(const DevLayout &d, int len, int maxlen, int from,
                                                  int64_t b, double r) {
    const int lane = threadIdx.x & 31;
    for (int t = from; t < maxlen; ++t) {
        const bool act = len > t;
        const unsigned m = __ballot_sync(kFull, act);
        if (act) {
            const int32_t k = d.rows[b + lane];
            d.E[k] *= r;
        }
        b += __popc(m);
    }
}

struct SharedState {
    double wa[kMaxWarps];
    double wb[kMaxWarps];
    double db;
    double G, H;
    int ok;
};

// Phase A + all-reduce for column j on this CTA's slice.  Returns false on abort.
// On return (all threads) sh.G, sh.H hold the grid totals.
__device__ bool column_reduce(const DevLayout &d, int j, unsigned long long seq, long long timeout_ns,
                              SharedState &sh, LaneCache &lc, bool &have_lc) {
    const int s = blockIdx.x;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const int64_t so = static_cast<int64_t>(s) * (d.J + 1) + j;
    const int64_t seg0 = d.slice_seg[so], seg1 = d.slice_seg[so + 1];
    const int64_t grp0 = d.slice_grp[so];
    const int ngrp = static_cast<int>((seg1 - seg0 + 31) >> 5);
    double G = 0.0, H = 0.0;
    have_lc = false;
    double *stash = d.stash + 2 * static_cast<int64_t>(s) * d.stash_stride;
    for (int g = warp; g < ngrp; g += nwarps) {
        const int64_t si = seg0 + 32 * static_cast<int64_t>(g) + lane;
        const int64_t base = d.grp_base[grp0 + g];
        if (g == warp) {
            group_phase_a(d, si, seg1, base, G, H, &lc, nullptr);
            have_lc = true;
        } else {
            group_phase_a(d, si, seg1, base, G, H, nullptr, stash + 2 * (si - seg0));
        }
    }
    G = warp_sum_lane0(G);
    H = warp_sum_lane0(H);
    if (lane == 0) {
        sh.wa[warp] = G;
        sh.wb[warp] = H;
    }
    __syncthreads();
    if (warp == 0) {
        double a = lane < nwarps ? sh.wa[lane] : 0.0;
        double b = lane < nwarps ? sh.wb[lane] : 0.0;
        a = __shfl_sync(kFull, warp_sum_lane0(a), 0);
        b = __shfl_sync(kFull, warp_sum_lane0(b), 0);
        double At, Bt;
        const bool ok = grid_allreduce2(d, seq, a, b, At, Bt, timeout_ns);
        if (lane == 0) {
            sh.ok = ok;
            sh.G = At;
            sh.H = Bt;
        }
    }
    __syncthreads();
    return sh.ok != 0;
}

// Phase C for column j with ratio r = e^{db} and em1 = e^{db} - 1.
__device__ void column_update(const DevLayout &d, int j, double r, double em1, const LaneCache &lc,
                              bool have_lc) {
    const int s = blockIdx.x;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const int64_t so = static_cast<int64_t>(s) * (d.J + 1) + j;
    const int64_t seg0 = d.slice_seg[so], seg1 = d.slice_seg[so + 1];
    const int64_t grp0 = d.slice_grp[so];
    const int ngrp = static_cast<int>((seg1 - seg0 + 31) >> 5);
    const double *stash = d.stash + 2 * static_cast<int64_t>(s) * d.stash_stride;
    if (have_lc) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (lc.row[u] >= 0) d.E[lc.row[u]] = lc.e[u] * r;
        if (lc.pid >= 0) d.D[lc.pid] = lc.Dv + em1 * lc.num;
        const int maxlen = __shfl_sync(kFull, lc.len, 0);
        if (maxlen > kUnroll) group_tail_update(d, lc.len, maxlen, kUnroll, lc.tail_base, r);
    }
    for (int g = warp + nwarps; g < ngrp; g += nwarps) {
        const int64_t si = seg0 + 32 * static_cast<int64_t>(g) + lane;
        const bool valid = si < seg1;
        const int2 sg = valid ? d.segs[si] : make_int2(0, 0);
        const int maxlen = __shfl_sync(kFull, sg.y, 0);
        group_tail_update(d, sg.y, maxlen, 0, d.grp_base[grp0 + g], r);
        if (valid) {
            const double num = stash[2 * (si - seg0)];
            const double Dv = stash[2 * (si - seg0) + 1];
            d.D[sg.x] = Dv + em1 * num;
        }
    }
}

// Recompute D_i = sum_{k in i} E_k on this CTA's subjects and return (in sh.G, sh.H after
// the all-reduce) the totals of the positive and negative parts of sum_i n_i log D_i.
__device__ bool refresh_and_reduce(const DevLayout &d, unsigned long long seq, long long timeout_ns,
                                   SharedState &sh, bool refresh) {
    const int s = blockIdx.x;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const int64_t p0 = d.shard_pat[s], p1 = d.shard_pat[s + 1];
    double pos = 0.0, neg = 0.0;
    for (int64_t i = p0 + threadIdx.x; i < p1; i += blockDim.x) {
        double Di;
        if (refresh) {
            Di = 0.0;
#pragma unroll 4
            for (int64_t k = d.pat_ptr[i]; k < d.pat_ptr[i + 1]; ++k) Di += d.E[k];
            d.D[i] = Di;
        } else {
            Di = d.D[i];
        }
        const double t = static_cast<double>(d.nev[i]) * log(Di);
        if (t >= 0.0) pos += t; else neg -= t;  // a NaN lands in neg and stays visible
    }
    pos = warp_sum_lane0(pos);
    neg = warp_sum_lane0(neg);
    if (lane == 0) {
        sh.wa[warp] = pos;
        sh.wb[warp] = neg;
    }
    __syncthreads();
    if (warp == 0) {
        double a = lane < nwarps ? sh.wa[lane] : 0.0;
        double b = lane < nwarps ? sh.wb[lane] : 0.0;
        a = __shfl_sync(kFull, warp_sum_lane0(a), 0);
        b = __shfl_sync(kFull, warp_sum_lane0(b), 0);
        double At, Bt;
        const bool ok = grid_allreduce2(d, seq, a, b, At, Bt, timeout_ns);
        if (lane == 0) {
            sh.ok = ok;
            sh.G = At;
            sh.H = Bt;
        }
    }
    __syncthreads();
    return sh.ok != 0;
}

// sum_j b_j Y'X_j (= Y'Xb) and the prior term, from this CTA's private beta, in j order.
__device__ void beta_terms(const DevLayout &d, const FitParams &p, double &lin, double &logprior) {
    const double *beta = d.beta_priv + static_cast<int64_t>(blockIdx.x) * d.J;
    double l = 0.0, sq = 0.0, ab = 0.0;
    for (int j = 0; j < d.J; ++j) {
        const double b = beta[j];
        l += b * d.ytx[j];
        sq += b * b;
        ab += fabs(b);
    }
    lin = l;
    logprior = p.prior == 1 ? -sq / (2.0 * p.variance) : (p.prior == 2 ? -p.lambda * ab : 0.0);
}

__global__ void __launch_bounds__(512, 1) fit_kernel(DevLayout d, FitParams p, FitOut *out, double *hist) {
    __shared__ SharedState sh;
    __shared__ int sh_stop;
    const int s = blockIdx.x;
    const bool leader = (s == 0) && (threadIdx.x == 0);
    const long long timeout = p.timeout_ns;
    unsigned long long seq = p.seq0;
    double *beta = d.beta_priv + static_cast<int64_t>(s) * d.J;
    double *trust = d.trust_priv + static_cast<int64_t>(s) * d.J;

    // P at the start point.
    if (!refresh_and_reduce(d, seq++, timeout, sh, true)) goto aborted;
    {
        double lin = 0.0, lp = 0.0;
        if (threadIdx.x == 0) beta_terms(d, p, lin, lp);
        double P_prev = lin - (sh.G - sh.H) + lp;
        if (leader && p.record_history) hist[0] = P_prev;
        int status = kStNotConverged, warn = 0, cycles = 0;
        long long nonzero = 0;
        double conv = 0.0, P = P_prev, loglik = lin - (sh.G - sh.H);
        if (!(P_prev == P_prev) || isinf(P_prev)) status = kStNumeric;
        for (int c = 1; c <= p.max_cycles && status == kStNotConverged; ++c) {
            double lin_c = 0.0, sq_c = 0.0, ab_c = 0.0;
            for (int j = 0; j < d.J; ++j) {
                LaneCache lc;
                bool have_lc;
                if (!column_reduce(d, j, seq++, timeout, sh, lc, have_lc)) goto aborted;
                if (threadIdx.x == 0) {
                    const double g = d.ytx[j] - sh.G;
                    const double h = -sh.H;
                    const double bj = beta[j];
                    double tr = trust[j];
                    double db = newton_step(g, h, bj, p.prior, p.variance, p.lambda, tr, warn);
                    if (!(db == db) || isinf(db)) {
                        db = 0.0;
                        status = kStNumeric;
                    }
                    const double nb = bj + db;
                    beta[j] = nb;
                    trust[j] = tr;
                    lin_c += nb * d.ytx[j];
                    sq_c += nb * nb;
                    ab_c += fabs(nb);
                    if (db != 0.0) ++nonzero;
                    sh.db = db;
                }
                __syncthreads();
                const double db = sh.db;
                if (db != 0.0) column_update(d, j, exp(db), expm1(db), lc, have_lc);
                __syncthreads();
            }
            if (!refresh_and_reduce(d, seq++, timeout, sh, true)) goto aborted;
            if (threadIdx.x == 0) {
                const double lp = p.prior == 1 ? -sq_c / (2.0 * p.variance)
                                               : (p.prior == 2 ? -p.lambda * ab_c : 0.0);
                loglik = lin_c - (sh.G - sh.H);
                P = loglik + lp;
                if (leader && p.record_history) hist[c] = P;
                conv = fabs(P - P_prev);
                if (p.tol_mode == 1) conv /= fmax(1.0, fabs(P));
                cycles = c;
                if (!(P == P) || isinf(P)) status = kStNumeric;
                else if (status == kStNotConverged && p.tol >= 0.0 && conv < p.tol) status = kStOk;
                P_prev = P;
                sh_stop = status;
            }
            __syncthreads();
            status = sh_stop;
        }
        if (leader) {
            out->logpost = P;
            out->loglik = loglik;
            out->conv = conv;
            out->cycles = cycles;
            out->status = status;
            out->nonzero_steps = nonzero;
            out->warnings = warn;
            out->seq_end = seq;
            out->err_where = 0;
        }
        return;
    }
aborted:
    if (threadIdx.x == 0) {
        if (s == 0) {
            out->status = kStTimeout;
            out->err_where = 1;
        }
    }
}

__global__ void __launch_bounds__(512, 1) grad_hess_kernel(DevLayout d, int j, FitParams p, FitOut *out) {
    __shared__ SharedState sh;
    const long long timeout = p.timeout_ns;
    unsigned long long seq = p.seq0;
    if (!refresh_and_reduce(d, seq++, timeout, sh, true)) goto aborted;
    {
        LaneCache lc;
        bool have_lc;
        if (!column_reduce(d, j, seq++, timeout, sh, lc, have_lc)) goto aborted;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            out->g = d.ytx[j] - sh.G;
            out->h = -sh.H;
            out->status = kStOk;
            out->seq_end = seq;
        }
        return;
    }
aborted:
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out->status = kStTimeout;
        out->err_where = 2;
    }
}

// E_k = l_k exp(Xb_k) on this CTA's rows, with Xb accumulated column by column in j order;
// private beta copies and trust radii (= 1) are (re)set.
__global__ void __launch_bounds__(512, 1) init_state_kernel(DevLayout d, const double *beta0) {
    const int s = blockIdx.x;
    const int64_t r0 = d.shard_row[s], r1 = d.shard_row[s + 1];
    double *beta = d.beta_priv + static_cast<int64_t>(s) * d.J;
    double *trust = d.trust_priv + static_cast<int64_t>(s) * d.J;
    for (int j = threadIdx.x; j < d.J; j += blockDim.x) {
        beta[j] = beta0 ? beta0[j] : 0.0;
        trust[j] = 1.0;
    }
    if (!beta0) {
        for (int64_t k = r0 + threadIdx.x; k < r1; k += blockDim.x) d.E[k] = d.L[k];
        return;
    }
    for (int64_t k = r0 + threadIdx.x; k < r1; k += blockDim.x) d.E[k] = 0.0;
    __syncthreads();
    for (int j = 0; j < d.J; ++j) {
        const double bj = beta0[j];
        if (bj == 0.0) continue;
        const int64_t so = static_cast<int64_t>(s) * (d.J + 1) + j;
        for (int64_t q = d.slice_row[so] + threadIdx.x; q < d.slice_row[so + 1]; q += blockDim.x)
            d.E[d.rows[q]] += bj;
        __syncthreads();
    }
    for (int64_t k = r0 + threadIdx.x; k < r1; k += blockDim.x) d.E[k] = d.L[k] * exp(d.E[k]);
}

}  // namespace

int launch_init_state(const DevLayout &d, const double *beta0_dev, int threads, void *stream) {
    init_state_kernel<<<d.S, threads, 0, static_cast<cudaStream_t>(stream)>>>(d, beta0_dev);
    return static_cast<int>(cudaGetLastError());
}

int launch_fit(const DevLayout &d, const FitParams &p, FitOut *out_dev, double *hist_dev, int threads,
               void *stream) {
    DevLayout dd = d;
    FitParams pp = p;
    void *args[] = {&dd, &pp, &out_dev, &hist_dev};
    return static_cast<int>(cudaLaunchCooperativeKernel(reinterpret_cast<void *>(fit_kernel), dim3(d.S),
                                                         dim3(threads), args, 0,
                                                         static_cast<cudaStream_t>(stream)));
}

int launch_grad_hess(const DevLayout &d, int32_t j, const FitParams &p, FitOut *out_dev, int threads,
                     void *stream) {
    DevLayout dd = d;
    FitParams pp = p;
    int jj = j;
    void *args[] = {&dd, &jj, &pp, &out_dev};
    return static_cast<int>(cudaLaunchCooperativeKernel(reinterpret_cast<void *>(grad_hess_kernel),
                                                         dim3(d.S), dim3(threads), args, 0,
                                                         static_cast<cudaStream_t>(stream)));
}

int launch_grad_hess_partial(const DevLayout &d, int32_t j, const FitParams &p, FitOut *out_dev,
                             int threads, int ctas, void *stream) {
    DevLayout dd = d;
    FitParams pp = p;
    int jj = j;
    void *args[] = {&dd, &jj, &pp, &out_dev};
    return static_cast<int>(cudaLaunchCooperativeKernel(reinterpret_cast<void *>(grad_hess_kernel),
                                                         dim3(ctas), dim3(threads), args, 0,
                                                         static_cast<cudaStream_t>(stream)));
}

int fit_kernel_max_blocks_per_sm(int threads, int *blocks) {
    int a = 0, b = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, fit_kernel, threads, 0);
    if (e != cudaSuccess) return static_cast<int>(e);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, grad_hess_kernel, threads, 0);
    if (e != cudaSuccess) return static_cast<int>(e);
    *blocks = a < b ? a : b;
    return 0;
}

}  // namespace sccs
