// sccs_host.cpp -- C ABI of the BSCCS library: input validation, canonical layout, device
// memory, and the host side of fit / gradient / log-posterior calls.
//
// Canonical form (Section 2.3 "Representation in Memory" of arXiv 1208.0945):
//   - subjects with n_i = 0 removed (they contribute nothing, Section 2.1);
//   - X in compressed column storage with rows ascending, ones implicit;
//   - the kept rows cut into S shards at subject boundaries, balanced by row count;
//   - each column's per-shard slice stored as subject segments (the COO form of M X_j),
//     longest first, 32 per group, rows diagonal-major inside a group.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "sccs.h"
#include "sccs_internal.h"

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(SCCS_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

constexpr long long kDefaultWaitNs = 2000000000LL;  // 2 s per device-side wait
// SCCS_PREC_FP32_POLISH: the FP32 phase stops at this relative change of the log-posterior
// (about what FP32 arithmetic can still resolve); the FP64 polish takes it from there.
constexpr double kFp32PhaseRelTol = 1e-6;

// Run f(t) for t in [0, n) on up to hardware_concurrency threads.
template <class F>
void parallel_for(int64_t n, F f) {
    unsigned hw = std::thread::hardware_concurrency();
    int64_t T = std::max<int64_t>(1, std::min<int64_t>(hw ? hw : 4, n));
    if (T <= 1) {
        for (int64_t i = 0; i < n; ++i) f(i);
        return;
    }
    std::atomic<int64_t> next(0);
    std::vector<std::thread> pool;
    for (int64_t t = 0; t < T; ++t)
        pool.emplace_back([&]() {
            for (;;) {
                int64_t i = next.fetch_add(1);
                if (i >= n) break;
                f(i);
            }
        });
    for (auto &th : pool) th.join();
}

struct DeviceArena {
    sccs_alloc_fn alloc = nullptr;
    sccs_free_fn free = nullptr;
    void *ctx = nullptr;
    struct Block {
        void *p;
        size_t bytes;
    };
    std::vector<Block> blocks;
    int64_t total = 0;
    int64_t uploaded = 0;

    void *get(size_t bytes) {
        size_t b = std::max<size_t>(bytes, 16);
        void *p = nullptr;
        if (alloc) {
            p = alloc(b, ctx);
        } else if (cudaMalloc(&p, b) != cudaSuccess) {
            (void)cudaGetLastError();
            p = nullptr;
        }
        if (p) {
            blocks.push_back({p, b});
            total += static_cast<int64_t>(b);
        }
        return p;
    }
    void release_all() {
        for (auto &blk : blocks) {
            if (free) free(blk.p, blk.bytes, ctx);
            else cudaFree(blk.p);
        }
        blocks.clear();
        total = 0;
    }
};

}  // namespace

struct sccs_handle {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int threads = 512;
    DeviceArena arena;
    sccs::DevLayout d{};
    int32_t prior = SCCS_PRIOR_NONE;
    double variance = 1.0;
    unsigned long long seq = 0;
    sccs::FitOut *out_dev = nullptr;
    sccs::FitOut *out_host = nullptr;  // pinned
    double *hist_dev = nullptr;
    int32_t hist_cap = 0;
    double *beta_dev = nullptr;        // J, scratch for start points
    double *hist_host = nullptr;       // pinned, hist_cap
    double *beta_host = nullptr;       // pinned, J
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    sccs_data_info info{};
};

namespace {

int set_device(const sccs_handle *h) {
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    return SCCS_OK;
}

// Copy `count` elements to a new device array; `pad` zeroed bytes follow them (arrays read
// by bulk copies rounded out to 16-byte boundaries).
template <class T>
int upload(sccs_handle *h, T **dst, const T *src, size_t count, size_t pad = 0) {
    *dst = static_cast<T *>(h->arena.get(count * sizeof(T) + pad));
    if (!*dst) return fail(SCCS_E_NOMEM, "device allocation failed");
    if (pad) {
        cudaError_t e = cudaMemsetAsync(reinterpret_cast<char *>(*dst) + count * sizeof(T), 0, pad, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    }
    if (count) {
        cudaError_t e = cudaMemcpyAsync(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync H2D");
        h->arena.uploaded += static_cast<int64_t>(count * sizeof(T));
    }
    return SCCS_OK;
}

template <class T>
int alloc_zero(sccs_handle *h, T **dst, size_t count) {
    *dst = static_cast<T *>(h->arena.get(count * sizeof(T)));
    if (!*dst) return fail(SCCS_E_NOMEM, "device allocation failed");
    cudaError_t e = cudaMemsetAsync(*dst, 0, std::max<size_t>(count, 1) * sizeof(T), h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    return SCCS_OK;
}

void destroy_handle(sccs_handle *h) {
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    h->arena.release_all();
    if (h->out_host) cudaFreeHost(h->out_host);
    if (h->hist_host) cudaFreeHost(h->hist_host);
    if (h->beta_host) cudaFreeHost(h->beta_host);
    if (h->hist_dev) cudaFree(h->hist_dev);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

// Host-built canonical layout.
struct HostLayout {
    int64_t K = 0, N = 0, nnz = 0;
    int32_t J = 0, S = 0;
    std::vector<int64_t> pat_ptr;   // N+1
    std::vector<int32_t> nev;       // N
    std::vector<double> L;          // K
    std::vector<double> ytx;        // J
    std::vector<int64_t> shard_row, shard_pat;
    std::vector<int32_t> rows;      // JDS rows
    std::vector<int2> segs;
    std::vector<int64_t> grp_base;
    std::vector<int64_t> slice_row, slice_seg, slice_grp;  // S*(J+1)
    int64_t stash_stride = 1;
    int64_t segments = 0;
    int64_t max_col = 0;
    int64_t subjects_in = 0;
};

// Checks everything about the inputs that needs no GPU.
int validate_inputs(int64_t K, const int64_t *patient_id, const int32_t *y, const double *Lin, int32_t J,
                    const int64_t *col_ptr, const int32_t *row_idx, const double *x_values) {
    if (K < 0 || J < 0) return fail(SCCS_E_INVAL, "K and J must be >= 0");
    if (K > 0 && (!patient_id || !y || !Lin)) return fail(SCCS_E_INVAL, "null row array");
    if (!col_ptr) return fail(SCCS_E_INVAL, "col_ptr is null");
    if (col_ptr[0] != 0) return fail(SCCS_E_INVAL, "col_ptr[0] must be 0");
    for (int32_t j = 0; j < J; ++j)
        if (col_ptr[j + 1] < col_ptr[j]) return fail(SCCS_E_INVAL, "col_ptr decreases at column " + std::to_string(j));
    const int64_t nnz_in = col_ptr[J];
    if (nnz_in > 0 && !row_idx) return fail(SCCS_E_INVAL, "row_idx is null");
    for (int64_t k = 1; k < K; ++k)
        if (patient_id[k] < patient_id[k - 1])
            return fail(SCCS_E_UNSORTED, "patient_id decreases at row " + std::to_string(k));
    for (int64_t k = 0; k < K; ++k) {
        if (y[k] < 0) return fail(SCCS_E_INVAL, "negative event count at row " + std::to_string(k));
        if (!(Lin[k] > 0.0) || !std::isfinite(Lin[k]))
            return fail(SCCS_E_INVAL, "offset must be positive and finite at row " + std::to_string(k));
    }
    for (int64_t e = 0; e < nnz_in; ++e)
        if (row_idx[e] < 0 || static_cast<int64_t>(row_idx[e]) >= K)
            return fail(SCCS_E_INVAL, "row index out of range at nonzero " + std::to_string(e));
    if (x_values)
        for (int64_t e = 0; e < nnz_in; ++e)
            if (x_values[e] != 1.0)
                return fail(SCCS_E_NONBINARY, "X value at nonzero " + std::to_string(e) + " is not 1");
    return SCCS_OK;
}

int build_layout(int64_t K, const int64_t *patient_id, const int32_t *y, const double *Lin, int32_t J,
                 const int64_t *col_ptr, const int32_t *row_idx, int32_t S, HostLayout &hl) {
    // ---- subjects, n_i, dropping n_i = 0
    std::vector<int64_t> sub_start;
    std::vector<int64_t> sub_n;
    for (int64_t k = 0; k < K; ++k) {
        if (k == 0 || patient_id[k] != patient_id[k - 1]) {
            sub_start.push_back(k);
            sub_n.push_back(0);
        }
        sub_n.back() += y[k];
    }
    const int64_t nsub = static_cast<int64_t>(sub_start.size());
    sub_start.push_back(K);
    hl.subjects_in = nsub;
    std::vector<int32_t> newrow(static_cast<size_t>(K), -1);
    int64_t Kk = 0, Nk = 0;
    for (int64_t i = 0; i < nsub; ++i)
        if (sub_n[i] > 0) {
            Kk += sub_start[i + 1] - sub_start[i];
            Nk++;
        }
    if (Kk >= (int64_t(1) << 31)) return fail(SCCS_E_INVAL, "more than 2^31-1 kept rows");
    for (int64_t i = 0; i < nsub; ++i)
        if (sub_n[i] >= (int64_t(1) << 31)) return fail(SCCS_E_INVAL, "n_i exceeds 2^31-1");
    hl.K = Kk;
    hl.N = Nk;
    hl.J = J;
    hl.pat_ptr.assign(static_cast<size_t>(Nk) + 1, 0);
    hl.nev.assign(static_cast<size_t>(Nk), 0);
    hl.L.assign(static_cast<size_t>(Kk), 0.0);
    std::vector<int32_t> row_pat(static_cast<size_t>(Kk));
    std::vector<int64_t> ykept(static_cast<size_t>(Kk));
    {
        int64_t i2 = 0, k2 = 0;
        for (int64_t i = 0; i < nsub; ++i) {
            if (sub_n[i] == 0) continue;
            hl.pat_ptr[i2] = k2;
            hl.nev[i2] = static_cast<int32_t>(sub_n[i]);
            for (int64_t k = sub_start[i]; k < sub_start[i + 1]; ++k) {
                newrow[k] = static_cast<int32_t>(k2);
                row_pat[k2] = static_cast<int32_t>(i2);
                hl.L[k2] = Lin[k];
                ykept[k2] = y[k];
                k2++;
            }
            i2++;
        }
        hl.pat_ptr[Nk] = Kk;
    }

    // ---- columns: map, drop, sort, reject duplicates; Y'X_j
    std::vector<int64_t> cptr(static_cast<size_t>(J) + 1, 0);
    {
        std::vector<int64_t> cnt(static_cast<size_t>(J), 0);
        parallel_for(J, [&](int64_t j) {
            int64_t c = 0;
            for (int64_t e = col_ptr[j]; e < col_ptr[j + 1]; ++e) c += newrow[row_idx[e]] >= 0;
            cnt[j] = c;
        });
        for (int32_t j = 0; j < J; ++j) cptr[j + 1] = cptr[j] + cnt[j];
    }
    hl.nnz = cptr[J];
    std::vector<int32_t> crow(static_cast<size_t>(hl.nnz));
    std::vector<int> dup(static_cast<size_t>(J), 0);
    hl.ytx.assign(static_cast<size_t>(J), 0.0);
    parallel_for(J, [&](int64_t j) {
        int64_t w = cptr[j];
        for (int64_t e = col_ptr[j]; e < col_ptr[j + 1]; ++e) {
            int32_t r = newrow[row_idx[e]];
            if (r >= 0) crow[w++] = r;
        }
        std::sort(crow.begin() + cptr[j], crow.begin() + cptr[j + 1]);
        int64_t t = 0;
        for (int64_t e = cptr[j]; e < cptr[j + 1]; ++e) {
            if (e > cptr[j] && crow[e] == crow[e - 1]) dup[j] = 1;
            t += ykept[crow[e]];
        }
        hl.ytx[j] = static_cast<double>(t);
    });
    for (int32_t j = 0; j < J; ++j)
        if (dup[j]) return fail(SCCS_E_DUPLICATE, "a row appears twice in column " + std::to_string(j));
    for (int32_t j = 0; j < J; ++j) hl.max_col = std::max<int64_t>(hl.max_col, cptr[j + 1] - cptr[j]);

    // ---- shards at subject boundaries, balanced by rows
    hl.S = S;
    hl.shard_pat.assign(static_cast<size_t>(S) + 1, 0);
    hl.shard_row.assign(static_cast<size_t>(S) + 1, 0);
    for (int32_t s = 1; s < S; ++s) {
        const int64_t target = (Kk * s) / S;
        const int64_t p = std::lower_bound(hl.pat_ptr.begin(), hl.pat_ptr.end(), target) - hl.pat_ptr.begin();
        hl.shard_pat[s] = std::max<int64_t>(hl.shard_pat[s - 1], std::min<int64_t>(p, Nk));
    }
    hl.shard_pat[S] = Nk;
    for (int32_t s = 0; s <= S; ++s) hl.shard_row[s] = hl.pat_ptr[hl.shard_pat[s]];

    // ---- pass 1: per (shard, column) slice: nonzeros and segments
    const int64_t SJ = static_cast<int64_t>(S) * (J + 1);
    std::vector<int64_t> s_nnz(static_cast<size_t>(SJ), 0), s_seg(static_cast<size_t>(SJ), 0);
    std::vector<int64_t> s_lo(static_cast<size_t>(SJ), 0);
    parallel_for(S, [&](int64_t s) {
        const int32_t r0 = static_cast<int32_t>(hl.shard_row[s]), r1 = static_cast<int32_t>(hl.shard_row[s + 1]);
        for (int32_t j = 0; j < J; ++j) {
            auto b = crow.begin() + cptr[j], e = crow.begin() + cptr[j + 1];
            auto lo = std::lower_bound(b, e, r0), hi = std::lower_bound(b, e, r1);
            const int64_t idx = s * (J + 1) + j;
            s_lo[idx] = lo - crow.begin();
            s_nnz[idx] = hi - lo;
            int64_t ns = 0;
            int32_t prev = -1;
            for (auto it = lo; it != hi; ++it) {
                const int32_t p = row_pat[*it];
                if (p != prev) {
                    ns++;
                    prev = p;
                }
            }
            s_seg[idx] = ns;
        }
    });
    hl.slice_row.assign(static_cast<size_t>(SJ), 0);
    hl.slice_seg.assign(static_cast<size_t>(SJ), 0);
    hl.slice_grp.assign(static_cast<size_t>(SJ), 0);
    int64_t tr = 0, ts = 0, tg = 0;
    int64_t max_seg = 1;
    for (int32_t s = 0; s < S; ++s) {
        for (int32_t j = 0; j <= J; ++j) {
            const int64_t idx = static_cast<int64_t>(s) * (J + 1) + j;
            hl.slice_row[idx] = tr;
            hl.slice_seg[idx] = ts;
            hl.slice_grp[idx] = tg;
            if (j < J) {
                tr += s_nnz[idx];
                ts += s_seg[idx];
                tg += (s_seg[idx] + 31) / 32;
                max_seg = std::max<int64_t>(max_seg, s_seg[idx]);
            }
        }
    }
    hl.stash_stride = max_seg;
    hl.segments = ts;
    hl.rows.assign(static_cast<size_t>(tr), 0);
    hl.segs.assign(static_cast<size_t>(ts), int2{0, 0});
    hl.grp_base.assign(static_cast<size_t>(tg), 0);

    // ---- pass 2: fill segments (longest first) and rows (diagonal-major per group)
    parallel_for(S, [&](int64_t s) {
        std::vector<int64_t> seg_start;
        std::vector<int32_t> seg_len, seg_pid, order;
        for (int32_t j = 0; j < J; ++j) {
            const int64_t idx = s * (J + 1) + j;
            const int64_t lo = s_lo[idx], n = s_nnz[idx];
            seg_start.clear();
            seg_len.clear();
            seg_pid.clear();
            int32_t prev = -1;
            for (int64_t q = lo; q < lo + n; ++q) {
                const int32_t p = row_pat[crow[q]];
                if (p != prev) {
                    seg_start.push_back(q);
                    seg_len.push_back(0);
                    seg_pid.push_back(p);
                    prev = p;
                }
                seg_len.back()++;
            }
            const int32_t ns = static_cast<int32_t>(seg_len.size());
            order.resize(ns);
            for (int32_t i = 0; i < ns; ++i) order[i] = i;
            std::stable_sort(order.begin(), order.end(),
                             [&](int32_t a, int32_t b) { return seg_len[a] > seg_len[b]; });
            int64_t rpos = hl.slice_row[idx];
            const int64_t spos = hl.slice_seg[idx], gpos = hl.slice_grp[idx];
            for (int32_t i = 0; i < ns; ++i) hl.segs[spos + i] = int2{seg_pid[order[i]], seg_len[order[i]]};
            for (int32_t g = 0; g * 32 < ns; ++g) {
                hl.grp_base[gpos + g] = rpos;
                const int32_t a = g * 32, b = std::min(ns, a + 32);
                const int32_t maxlen = seg_len[order[a]];
                for (int32_t t = 0; t < maxlen; ++t)
                    for (int32_t l = a; l < b; ++l) {
                        const int32_t o = order[l];
                        if (seg_len[o] > t) hl.rows[rpos++] = crow[seg_start[o] + t];
                    }
            }
        }
    });
    return SCCS_OK;
}

int run_init_state(sccs_handle *h, const double *beta_dev) {
    int e = sccs::launch_init_state(h->d, beta_dev, h->threads, h->stream);
    if (e != 0) return cuda_fail(static_cast<cudaError_t>(e), "init_state launch");
    return SCCS_OK;
}

// After an aborted kernel: clear the all-reduce slots and the abort flag, restart the
// sequence, and put the state back to beta = 0.
int reset_after_abort(sccs_handle *h) {
    cudaMemsetAsync(h->d.slots, 0, sizeof(unsigned long long) * 4 * static_cast<size_t>(h->d.S), h->stream);
    cudaMemsetAsync(h->d.abort_flag, 0, sizeof(int), h->stream);
    h->seq = 0;
    int rc = run_init_state(h, nullptr);
    cudaStreamSynchronize(h->stream);
    return rc;
}

int sync_out(sccs_handle *h) {
    cudaError_t e = cudaMemcpyAsync(h->out_host, h->out_dev, sizeof(sccs::FitOut), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync D2H");
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return SCCS_OK;
}

// Move the state to beta (host array) or leave it (nullptr).
int set_state(sccs_handle *h, const double *beta) {
    if (!beta) return SCCS_OK;
    const int32_t J = h->d.J;
    for (int32_t j = 0; j < J; ++j)
        if (!std::isfinite(beta[j])) return fail(SCCS_E_INVAL, "beta has a non-finite entry");
    std::memcpy(h->beta_host, beta, sizeof(double) * static_cast<size_t>(J));
    cudaError_t e = cudaMemcpyAsync(h->beta_dev, h->beta_host, sizeof(double) * std::max<int32_t>(J, 1),
                                    cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync beta");
    return run_init_state(h, h->beta_dev);
}

sccs::FitParams base_params(const sccs_handle *h) {
    sccs::FitParams p{};
    p.prior = h->prior;
    p.variance = h->variance;
    p.inv_var = 1.0 / h->variance;
    p.lambda = h->prior == SCCS_PRIOR_LAPLACE ? std::sqrt(2.0 / h->variance) : 0.0;
    p.tol_mode = SCCS_TOL_REL_LOGPOST;
    p.tol = 1e-12;
    p.max_cycles = 0;
    p.record_history = 0;
    p.seq0 = h->seq;
    p.timeout_ns = kDefaultWaitNs;
    return p;
}

// One launch of the fit kernel (FP64 or FP32 body) with its result checks; `ms` gets the
// kernel's event time.
int run_fit_phase(sccs_handle *h, const sccs::FitParams &p, bool fp32, sccs::FitOut &r, float &ms) {
    sccs::FitParams pp = p;
    pp.seq0 = h->seq;
    cudaEventRecord(h->ev0, h->stream);
    int le = sccs::launch_fit(h->d, pp, h->out_dev, h->hist_dev, h->threads, h->stream, fp32);
    if (le != 0) return cuda_fail(static_cast<cudaError_t>(le), "fit kernel launch");
    cudaEventRecord(h->ev1, h->stream);
    int rc = sync_out(h);
    if (rc) return rc;
    r = *h->out_host;
    if (r.status == -6 || r.abort_flag) {
        reset_after_abort(h);
        return fail(SCCS_E_TIMEOUT, "a device-side wait exceeded its bound; the handle was reset to beta = 0");
    }
    h->seq = r.seq_end;
    if (r.status == -7) {
        run_init_state(h, nullptr);
        cudaStreamSynchronize(h->stream);
        return fail(SCCS_E_NUMERIC, "non-finite gradient, step or log-posterior; the handle was reset to beta = 0");
    }
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    return SCCS_OK;
}

}  // namespace

bool sccs_handle_view(const sccs_handle *h, sccs::HandleView *v) {
    if (!h || !v) return false;
    v->device = h->device;
    v->threads = h->threads;
    v->d = h->d;
    return true;
}

extern "C" {

int sccs_set_error(int code, const char *msg) { return fail(code, msg ? msg : ""); }

int sccs_version(int32_t *abi_version, const char **build) {
    if (abi_version) *abi_version = SCCS_ABI_VERSION;
    if (build) *build = "sccs-gb300 sm_103a fp64";
    return SCCS_OK;
}

const char *sccs_last_error(const sccs_handle *) { return g_last_error.c_str(); }

int sccs_create(sccs_handle **out, int64_t K, const int64_t *patient_id, const int32_t *y,
                const double *offset_L, int32_t J, const int64_t *col_ptr, const int32_t *row_idx,
                const double *x_values, const sccs_create_opts *opts) {
    g_last_error.clear();
    if (!out) return fail(SCCS_E_INVAL, "out is null");
    *out = nullptr;
    sccs_create_opts o{};
    o.struct_size = sizeof(sccs_create_opts);
    if (opts) {
        if (opts->struct_size != static_cast<int32_t>(sizeof(sccs_create_opts)))
            return fail(SCCS_E_INVAL, "sccs_create_opts.struct_size mismatch");
        o = *opts;
    }
    int rcv = validate_inputs(K, patient_id, y, offset_L, J, col_ptr, row_idx, x_values);
    if (rcv != SCCS_OK) return rcv;
    int threads = o.threads_per_block ? o.threads_per_block : 512;
    if (threads < 64 || threads > 512 || threads % 32)
        return fail(SCCS_E_INVAL, "threads_per_block must be a multiple of 32 in [64, 512]");
    if ((o.alloc == nullptr) != (o.free == nullptr)) return fail(SCCS_E_INVAL, "alloc and free go together");

    cudaError_t ce = cudaSetDevice(o.device);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaSetDevice");
    int sms = 0;
    ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, o.device);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaDeviceGetAttribute");
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, o.device);
    if (!coop) return fail(SCCS_E_UNSUPPORTED, "device lacks cooperative launch");
    int per_sm = 0;
    int rc0 = sccs::fit_kernel_max_blocks_per_sm(threads, &per_sm);
    if (rc0 != 0) return cuda_fail(static_cast<cudaError_t>(rc0), "occupancy query");
    if (per_sm < 1) return fail(SCCS_E_UNSUPPORTED, "fit kernel does not fit on an SM");
    int S = o.num_shards ? o.num_shards : sms;
    if (S < 1 || S > sms * per_sm || S > sccs::kMaxShards)
        return fail(SCCS_E_INVAL, "num_shards must be in [1, " + std::to_string(std::min(sms * per_sm, sccs::kMaxShards)) + "]");

    HostLayout hl;
    int rc = build_layout(K, patient_id, y, offset_L, J, col_ptr, row_idx, S, hl);
    if (rc != SCCS_OK) return rc;

    sccs_handle *h = new sccs_handle();
    h->device = o.device;
    h->threads = threads;
    h->arena.alloc = o.alloc;
    h->arena.free = o.free;
    h->arena.ctx = o.alloc_ctx;
    if (o.stream) {
        h->stream = static_cast<cudaStream_t>(o.stream);
    } else {
        ce = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (ce != cudaSuccess) {
            delete h;
            return cuda_fail(ce, "cudaStreamCreate");
        }
        h->own_stream = true;
    }
    auto bail = [&](int code) {
        std::string msg = g_last_error;
        destroy_handle(h);
        g_last_error = msg;
        return code;
    };
    if ((ce = cudaEventCreate(&h->ev0)) != cudaSuccess || (ce = cudaEventCreate(&h->ev1)) != cudaSuccess)
        return bail(cuda_fail(ce, "cudaEventCreate"));
    if ((ce = cudaMallocHost(&h->out_host, sizeof(sccs::FitOut))) != cudaSuccess)
        return bail(cuda_fail(ce, "cudaMallocHost"));
    if ((ce = cudaMallocHost(&h->beta_host, sizeof(double) * std::max<int32_t>(J, 1))) != cudaSuccess)
        return bail(cuda_fail(ce, "cudaMallocHost"));

    sccs::DevLayout &d = h->d;
    d.S = S;
    d.J = J;
    d.K = hl.K;
    d.N = hl.N;
    int32_t *rows;
    int2 *segs;
    int64_t *grp_base, *slice_row, *slice_seg, *slice_grp, *shard_row, *shard_pat, *pat_ptr;
    int32_t *nev;
    double *L, *ytx;
    if ((rc = upload(h, &rows, hl.rows.data(), hl.rows.size(), sccs::kCopyPad)) ||
        (rc = upload(h, &segs, hl.segs.data(), hl.segs.size(), sccs::kCopyPad)) ||
        (rc = upload(h, &grp_base, hl.grp_base.data(), hl.grp_base.size(), sccs::kCopyPad)) ||
        (rc = upload(h, &slice_row, hl.slice_row.data(), hl.slice_row.size())) ||
        (rc = upload(h, &slice_seg, hl.slice_seg.data(), hl.slice_seg.size())) ||
        (rc = upload(h, &slice_grp, hl.slice_grp.data(), hl.slice_grp.size())) ||
        (rc = upload(h, &shard_row, hl.shard_row.data(), hl.shard_row.size())) ||
        (rc = upload(h, &shard_pat, hl.shard_pat.data(), hl.shard_pat.size())) ||
        (rc = upload(h, &pat_ptr, hl.pat_ptr.data(), hl.pat_ptr.size())) ||
        (rc = upload(h, &nev, hl.nev.data(), hl.nev.size())) ||
        (rc = upload(h, &L, hl.L.data(), hl.L.size())) ||
        (rc = upload(h, &ytx, hl.ytx.data(), hl.ytx.size())))
        return bail(rc);
    d.rows = rows;
    d.segs = segs;
    d.grp_base = grp_base;
    d.slice_row = slice_row;
    d.slice_seg = slice_seg;
    d.slice_grp = slice_grp;
    d.shard_row = shard_row;
    d.shard_pat = shard_pat;
    d.pat_ptr = pat_ptr;
    d.nev = nev;
    d.L = L;
    d.ytx = ytx;
    d.stash_stride = hl.stash_stride;
    if ((rc = alloc_zero(h, &d.E, static_cast<size_t>(hl.K))) ||
        (rc = alloc_zero(h, &d.D, static_cast<size_t>(hl.N))) ||
        (rc = alloc_zero(h, &d.E32, static_cast<size_t>(hl.K))) ||
        (rc = alloc_zero(h, &d.D32, static_cast<size_t>(hl.N))) ||
        (rc = alloc_zero(h, &d.beta_priv, static_cast<size_t>(S) * std::max<int32_t>(J, 1))) ||
        (rc = alloc_zero(h, &d.trust_priv, static_cast<size_t>(S) * std::max<int32_t>(J, 1))) ||
        (rc = alloc_zero(h, &d.stash, static_cast<size_t>(S) * 2 * static_cast<size_t>(hl.stash_stride))) ||
        (rc = alloc_zero(h, &d.slots, static_cast<size_t>(S) * 4)) ||
        (rc = alloc_zero(h, &h->out_dev, 1)) ||
        (rc = alloc_zero(h, &h->beta_dev, static_cast<size_t>(std::max<int32_t>(J, 1)))))
        return bail(rc);
    d.abort_flag = &h->out_dev->abort_flag;
    if ((rc = run_init_state(h, nullptr))) return bail(rc);
    ce = cudaStreamSynchronize(h->stream);
    if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaStreamSynchronize"));

    sccs_data_info &info = h->info;
    info.rows_in = K;
    info.rows_kept = hl.K;
    info.subjects_in = hl.subjects_in;
    info.subjects_kept = hl.N;
    info.nnz_kept = hl.nnz;
    info.segments = hl.segments;
    info.max_column_nnz = hl.max_col;
    info.device_bytes = h->arena.total;
    info.upload_bytes = h->arena.uploaded;
    info.columns = J;
    info.num_shards = S;
    info.threads_per_block = threads;
    *out = h;
    return SCCS_OK;
}

int sccs_destroy(sccs_handle *h) {
    destroy_handle(h);
    return SCCS_OK;
}

int sccs_get_info(const sccs_handle *h, sccs_data_info *info) {
    if (!h || !info) return fail(SCCS_E_INVAL, "null argument");
    *info = h->info;
    return SCCS_OK;
}

int sccs_set_prior(sccs_handle *h, int32_t prior_type, double variance) {
    if (!h) return fail(SCCS_E_INVAL, "null handle");
    if (prior_type != SCCS_PRIOR_NONE && prior_type != SCCS_PRIOR_NORMAL && prior_type != SCCS_PRIOR_LAPLACE)
        return fail(SCCS_E_INVAL, "unknown prior type");
    if (prior_type != SCCS_PRIOR_NONE && !(variance > 0.0 && std::isfinite(variance)))
        return fail(SCCS_E_INVAL, "prior variance must be positive and finite");
    h->prior = prior_type;
    h->variance = prior_type == SCCS_PRIOR_NONE ? 1.0 : variance;
    return SCCS_OK;
}

int sccs_fit(sccs_handle *h, const sccs_fit_opts *opts, double *beta_out, sccs_fit_info *info) {
    const auto t_start = std::chrono::steady_clock::now();
    if (!h) return fail(SCCS_E_INVAL, "null handle");
    sccs_fit_opts o{};
    o.struct_size = sizeof(sccs_fit_opts);
    o.tol_mode = SCCS_TOL_REL_LOGPOST;
    o.tol = 1e-12;
    o.max_cycles = 1000;
    o.precision = SCCS_PREC_FP64;
    if (opts) {
        if (opts->struct_size != static_cast<int32_t>(sizeof(sccs_fit_opts)))
            return fail(SCCS_E_INVAL, "sccs_fit_opts.struct_size mismatch");
        o = *opts;
    }
    if (o.max_cycles < 0) return fail(SCCS_E_INVAL, "max_cycles must be >= 0");
    if (o.tol_mode == SCCS_TOL_GENKIN_XBETA)
        return fail(SCCS_E_UNSUPPORTED, "the Genkin X-beta convergence test is not in this build");
    if (o.tol_mode != SCCS_TOL_ABS_LOGPOST && o.tol_mode != SCCS_TOL_REL_LOGPOST)
        return fail(SCCS_E_INVAL, "unknown tol_mode");
    if (o.precision != SCCS_PREC_FP64 && o.precision != SCCS_PREC_FP32_POLISH && o.precision != SCCS_PREC_FP32)
        return fail(SCCS_E_INVAL, "unknown precision");
    int rc = set_device(h);
    if (rc) return rc;

    // start point
    if (o.beta0) {
        if ((rc = set_state(h, o.beta0))) return rc;
    } else if (o.warm_start) {
        cudaError_t e = cudaMemcpyAsync(h->beta_dev, h->d.beta_priv, sizeof(double) * std::max<int32_t>(h->d.J, 1),
                                        cudaMemcpyDeviceToDevice, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync warm start");
        if ((rc = run_init_state(h, h->beta_dev))) return rc;
    } else {
        if ((rc = run_init_state(h, nullptr))) return rc;
    }
    const int32_t need = o.max_cycles + 1;
    if (need > h->hist_cap) {
        if (h->hist_dev) cudaFree(h->hist_dev);
        if (h->hist_host) cudaFreeHost(h->hist_host);
        h->hist_dev = nullptr;
        h->hist_host = nullptr;
        h->hist_cap = 0;
        cudaError_t e = cudaMalloc(&h->hist_dev, sizeof(double) * need);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc history");
        e = cudaMallocHost(&h->hist_host, sizeof(double) * need);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocHost history");
        h->hist_cap = need;
    }
    sccs::FitParams p = base_params(h);
    p.tol_mode = o.tol_mode;
    p.tol = o.tol;
    p.max_cycles = o.max_cycles;
    p.record_history = 1;

    sccs::FitOut r{};
    float ms = 0.f, ms32 = 0.f;
    int32_t fp32_cycles = 0;
    int64_t nonzero = 0;
    int32_t warnings = 0;
    if (o.precision != SCCS_PREC_FP64) {
        int le = sccs::launch_e_to_f32(h->d, h->threads, h->stream);
        if (le != 0) return cuda_fail(static_cast<cudaError_t>(le), "E conversion launch");
        sccs::FitParams p32 = p;
        if (o.precision == SCCS_PREC_FP32_POLISH) {
            // the FP32 phase always stops at its own switch point; the caller's tol (including
            // tol < 0, a fixed number of cycles) applies to the FP64 polish
            p32.tol_mode = SCCS_TOL_REL_LOGPOST;
            p32.tol = kFp32PhaseRelTol;
        }
        if ((rc = run_fit_phase(h, p32, true, r, ms32))) return rc;
        fp32_cycles = r.cycles;
        nonzero += r.nonzero_steps;
        warnings |= r.warnings;
        if (o.precision == SCCS_PREC_FP32_POLISH) {
            // FP64 polish from the FP32 point: E and D rebuilt in FP64 from beta, trust radii kept
            cudaError_t e = cudaMemcpyAsync(h->beta_dev, h->d.beta_priv, sizeof(double) * std::max<int32_t>(h->d.J, 1),
                                            cudaMemcpyDeviceToDevice, h->stream);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync polish start");
            le = sccs::launch_init_state(h->d, h->beta_dev, h->threads, h->stream, true);
            if (le != 0) return cuda_fail(static_cast<cudaError_t>(le), "init_state launch");
            if ((rc = run_fit_phase(h, p, false, r, ms))) return rc;
            nonzero += r.nonzero_steps;
            warnings |= r.warnings;
        }
    } else {
        if ((rc = run_fit_phase(h, p, false, r, ms))) return rc;
        nonzero = r.nonzero_steps;
        warnings = r.warnings;
    }
    if (beta_out && h->d.J > 0) {
        cudaError_t e = cudaMemcpy(beta_out, h->d.beta_priv, sizeof(double) * h->d.J, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "copy beta");
    }
    if (o.logpost_history) {
        cudaError_t e = cudaMemcpy(o.logpost_history, h->hist_dev, sizeof(double) * (r.cycles + 1),
                                   cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "copy history");
    }
    const int32_t total_cycles = o.precision == SCCS_PREC_FP32_POLISH ? fp32_cycles + r.cycles : r.cycles;
    if (info) {
        info->status = r.status;
        info->cycles = total_cycles;
        info->steps = static_cast<int64_t>(total_cycles) * h->d.J;
        info->nonzero_steps = nonzero;
        info->logpost = r.logpost;
        info->conv_value = r.conv;
        info->kernel_ms = ms + ms32;
        info->total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
        info->warnings = warnings;
        info->fp32_cycles = fp32_cycles;
    }
    return r.status == 0 ? SCCS_OK : SCCS_NOT_CONVERGED;
}

int sccs_fit_batch(sccs_handle *const *handles, int32_t n, const sccs_fit_opts *opts, double *const *beta_out,
                   sccs_fit_info *infos) {
    const auto t_start = std::chrono::steady_clock::now();
    if (n < 1 || !handles) return fail(SCCS_E_INVAL, "need at least one handle");
    sccs_fit_opts o{};
    o.struct_size = sizeof(sccs_fit_opts);
    o.tol_mode = SCCS_TOL_REL_LOGPOST;
    o.tol = 1e-12;
    o.max_cycles = 1000;
    o.precision = SCCS_PREC_FP64;
    if (opts) {
        if (opts->struct_size != static_cast<int32_t>(sizeof(sccs_fit_opts)))
            return fail(SCCS_E_INVAL, "sccs_fit_opts.struct_size mismatch");
        o = *opts;
    }
    if (o.beta0) return fail(SCCS_E_INVAL, "sccs_fit_batch takes no beta0 (use warm_start)");
    if (o.max_cycles < 0) return fail(SCCS_E_INVAL, "max_cycles must be >= 0");
    if (o.tol_mode != SCCS_TOL_ABS_LOGPOST && o.tol_mode != SCCS_TOL_REL_LOGPOST)
        return fail(o.tol_mode == SCCS_TOL_GENKIN_XBETA ? SCCS_E_UNSUPPORTED : SCCS_E_INVAL, "unsupported tol_mode");
    if (o.precision != SCCS_PREC_FP64 && o.precision != SCCS_PREC_FP32_POLISH && o.precision != SCCS_PREC_FP32)
        return fail(SCCS_E_INVAL, "unknown precision");
    for (int32_t k = 0; k < n; ++k) {
        if (!handles[k]) return fail(SCCS_E_INVAL, "null handle in batch");
        if (handles[k]->device != handles[0]->device) return fail(SCCS_E_INVAL, "handles on different devices");
        if (handles[k]->threads != handles[0]->threads) return fail(SCCS_E_INVAL, "handles with different threads_per_block");
        for (int32_t q = 0; q < k; ++q)
            if (handles[q] == handles[k]) return fail(SCCS_E_INVAL, "a handle appears twice in the batch");
    }
    sccs_handle *h0 = handles[0];
    int rc = set_device(h0);
    if (rc) return rc;
    const int threads = h0->threads;
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h0->device);
    if ((rc = sccs::fit_kernel_max_blocks_per_sm(threads, &per_sm))) return cuda_fail(static_cast<cudaError_t>(rc), "occupancy");
    const int capacity = sms * per_sm;
    cudaStream_t st = h0->stream;
    for (int32_t k = 0; k < n; ++k) {
        sccs_handle *h = handles[k];
        if (h->stream != st) cudaStreamSynchronize(h->stream);   // no work of the handle in flight elsewhere
        if (o.warm_start) {
            cudaMemcpyAsync(h->beta_dev, h->d.beta_priv, sizeof(double) * std::max<int32_t>(h->d.J, 1),
                            cudaMemcpyDeviceToDevice, st);
            if ((rc = sccs::launch_init_state(h->d, h->beta_dev, threads, st))) return cuda_fail(static_cast<cudaError_t>(rc), "init");
        } else if ((rc = sccs::launch_init_state(h->d, nullptr, threads, st))) {
            return cuda_fail(static_cast<cudaError_t>(rc), "init");
        }
        const int32_t need = o.max_cycles + 1;
        if (need > h->hist_cap) {
            if (h->hist_dev) cudaFree(h->hist_dev);
            if (h->hist_host) cudaFreeHost(h->hist_host);
            h->hist_dev = nullptr;
            h->hist_host = nullptr;
            h->hist_cap = 0;
            if (cudaMalloc(&h->hist_dev, sizeof(double) * need) != cudaSuccess ||
                cudaMallocHost(&h->hist_host, sizeof(double) * need) != cudaSuccess)
                return fail(SCCS_E_NOMEM, "history buffer");
            h->hist_cap = need;
        }
        if (h->d.S > capacity) return fail(SCCS_E_INVAL, "a handle has more shards than the device holds at once");
    }
    // waves of fits whose shard counts fit on the device together
    std::vector<std::vector<int32_t>> waves;
    {
        std::vector<int32_t> cur;
        int used = 0;
        for (int32_t k = 0; k < n; ++k) {
            if (used + handles[k]->d.S > capacity) {
                waves.push_back(cur);
                cur.clear();
                used = 0;
            }
            cur.push_back(k);
            used += handles[k]->d.S;
        }
        if (!cur.empty()) waves.push_back(cur);
    }
    sccs::BatchEntry *ent_dev = nullptr;
    int2 *map_dev = nullptr;
    if (cudaMalloc(&ent_dev, sizeof(sccs::BatchEntry) * n) != cudaSuccess ||
        cudaMalloc(&map_dev, sizeof(int2) * capacity) != cudaSuccess) {
        cudaFree(ent_dev);
        return fail(SCCS_E_NOMEM, "batch descriptors");
    }
    std::vector<sccs::BatchEntry> ent(n);
    std::vector<int2> map;
    std::vector<int> status(n, SCCS_OK);
    std::vector<sccs::FitOut> res(n);
    std::vector<int32_t> fp32_cycles(n, 0);
    std::vector<int64_t> nonzero(n, 0);
    std::vector<int32_t> warnings(n, 0);
    double kernel_ms = 0.0;
    auto run_phase = [&](bool fp32, bool polish_phase) -> int {
        for (int32_t k = 0; k < n; ++k) {
            sccs_handle *h = handles[k];
            sccs::FitParams p = base_params(h);
            p.tol_mode = o.tol_mode;
            p.tol = o.tol;
            p.max_cycles = o.max_cycles;
            p.record_history = 1;
            if (fp32 && o.precision == SCCS_PREC_FP32_POLISH) {
                p.tol_mode = SCCS_TOL_REL_LOGPOST;
                p.tol = kFp32PhaseRelTol;
            }
            ent[k] = sccs::BatchEntry{h->d, p, h->out_dev, h->hist_dev};
        }
        cudaMemcpyAsync(ent_dev, ent.data(), sizeof(sccs::BatchEntry) * n, cudaMemcpyHostToDevice, st);
        for (const auto &w : waves) {
            map.clear();
            for (int32_t k : w)
                for (int sidx = 0; sidx < handles[k]->d.S; ++sidx) map.push_back(make_int2(k, sidx));
            cudaMemcpyAsync(map_dev, map.data(), sizeof(int2) * map.size(), cudaMemcpyHostToDevice, st);
            cudaEventRecord(h0->ev0, st);
            int le = sccs::launch_fit_batch(ent_dev, map_dev, static_cast<int>(map.size()), threads, st, fp32);
            if (le != 0) return cuda_fail(static_cast<cudaError_t>(le), "batch kernel launch");
            cudaEventRecord(h0->ev1, st);
            cudaError_t e = cudaEventSynchronize(h0->ev1);
            if (e != cudaSuccess) return cuda_fail(e, "batch kernel");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, h0->ev0, h0->ev1);
            kernel_ms += ms;
        }
        for (int32_t k = 0; k < n; ++k)
            cudaMemcpyAsync(handles[k]->out_host, handles[k]->out_dev, sizeof(sccs::FitOut), cudaMemcpyDeviceToHost, st);
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "batch results");
        for (int32_t k = 0; k < n; ++k) {
            sccs_handle *h = handles[k];
            if (status[k] != SCCS_OK) continue;
            const sccs::FitOut r = *h->out_host;
            if (r.status == -6 || r.abort_flag) {
                reset_after_abort(h);
                status[k] = SCCS_E_TIMEOUT;
                continue;
            }
            h->seq = r.seq_end;
            if (r.status == -7) {
                run_init_state(h, nullptr);
                status[k] = SCCS_E_NUMERIC;
                continue;
            }
            res[k] = r;
            nonzero[k] += r.nonzero_steps;
            warnings[k] |= r.warnings;
            if (fp32) fp32_cycles[k] = r.cycles;
        }
        (void)polish_phase;
        return SCCS_OK;
    };
    auto done = [&](int code) {
        cudaFree(ent_dev);
        cudaFree(map_dev);
        return code;
    };
    if (o.precision != SCCS_PREC_FP64) {
        for (int32_t k = 0; k < n; ++k) {
            int le = sccs::launch_e_to_f32(handles[k]->d, threads, st);
            if (le != 0) return done(cuda_fail(static_cast<cudaError_t>(le), "E conversion launch"));
        }
        if ((rc = run_phase(true, false))) return done(rc);
        if (o.precision == SCCS_PREC_FP32_POLISH) {
            for (int32_t k = 0; k < n; ++k) {
                sccs_handle *h = handles[k];
                cudaMemcpyAsync(h->beta_dev, h->d.beta_priv, sizeof(double) * std::max<int32_t>(h->d.J, 1),
                                cudaMemcpyDeviceToDevice, st);
                int le = sccs::launch_init_state(h->d, h->beta_dev, threads, st, true);
                if (le != 0) return done(cuda_fail(static_cast<cudaError_t>(le), "init_state launch"));
            }
            if ((rc = run_phase(false, true))) return done(rc);
        }
    } else if ((rc = run_phase(false, false))) {
        return done(rc);
    }
    int first_err = SCCS_OK;
    for (int32_t k = 0; k < n; ++k) {
        sccs_handle *h = handles[k];
        const sccs::FitOut &r = res[k];
        if (status[k] == SCCS_OK && beta_out && beta_out[k] && h->d.J > 0) {
            cudaError_t e = cudaMemcpy(beta_out[k], h->d.beta_priv, sizeof(double) * h->d.J, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) status[k] = SCCS_E_CUDA;
        }
        if (infos) {
            sccs_fit_info &fi = infos[k];
            const int32_t cyc = o.precision == SCCS_PREC_FP32_POLISH ? fp32_cycles[k] + r.cycles : r.cycles;
            fi.status = status[k] != SCCS_OK ? status[k] : r.status;
            fi.cycles = cyc;
            fi.steps = static_cast<int64_t>(cyc) * h->d.J;
            fi.nonzero_steps = nonzero[k];
            fi.logpost = r.logpost;
            fi.conv_value = r.conv;
            fi.kernel_ms = kernel_ms;
            fi.total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
            fi.warnings = warnings[k];
            fi.fp32_cycles = fp32_cycles[k];
        }
        if (status[k] != SCCS_OK && first_err == SCCS_OK) first_err = status[k];
    }
    if (first_err != SCCS_OK) return done(fail(first_err, "at least one fit of the batch failed (see infos[k].status)"));
    return done(SCCS_OK);
}

int sccs_grad_hess(sccs_handle *h, int32_t j, const double *beta, double *g, double *hess) {
    if (!h) return fail(SCCS_E_INVAL, "null handle");
    if (j < 0 || j >= h->d.J) return fail(SCCS_E_INVAL, "column index out of range");
    int rc = set_device(h);
    if (rc) return rc;
    if ((rc = set_state(h, beta))) return rc;
    sccs::FitParams p = base_params(h);
    int le = sccs::launch_grad_hess(h->d, j, p, h->out_dev, h->threads, h->stream);
    if (le != 0) return cuda_fail(static_cast<cudaError_t>(le), "grad_hess kernel launch");
    if ((rc = sync_out(h))) return rc;
    const sccs::FitOut r = *h->out_host;
    if (r.status != 0 || r.abort_flag) {
        reset_after_abort(h);
        return fail(SCCS_E_TIMEOUT, "a device-side wait exceeded its bound; the handle was reset to beta = 0");
    }
    h->seq = r.seq_end;
    if (g) *g = r.g;
    if (hess) *hess = r.h;
    return SCCS_OK;
}

int sccs_logpost(sccs_handle *h, const double *beta, double *logpost, double *loglik) {
    if (!h) return fail(SCCS_E_INVAL, "null handle");
    int rc = set_device(h);
    if (rc) return rc;
    if ((rc = set_state(h, beta))) return rc;
    if (h->hist_cap < 1) {
        cudaError_t e = cudaMalloc(&h->hist_dev, sizeof(double));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc history");
        e = cudaMallocHost(&h->hist_host, sizeof(double));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocHost history");
        h->hist_cap = 1;
    }
    sccs::FitParams p = base_params(h);
    p.max_cycles = 0;
    int le = sccs::launch_fit(h->d, p, h->out_dev, h->hist_dev, h->threads, h->stream);
    if (le != 0) return cuda_fail(static_cast<cudaError_t>(le), "fit kernel launch");
    if ((rc = sync_out(h))) return rc;
    const sccs::FitOut r = *h->out_host;
    if (r.status == -6 || r.abort_flag) {
        reset_after_abort(h);
        return fail(SCCS_E_TIMEOUT, "a device-side wait exceeded its bound; the handle was reset to beta = 0");
    }
    h->seq = r.seq_end;
    if (logpost) *logpost = r.logpost;
    if (loglik) *loglik = r.loglik;
    return SCCS_OK;
}

int sccs_get_beta(const sccs_handle *h, double *beta_out) {
    if (!h || !beta_out) return fail(SCCS_E_INVAL, "null argument");
    if (h->d.J == 0) return SCCS_OK;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    e = cudaMemcpy(beta_out, h->d.beta_priv, sizeof(double) * h->d.J, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "copy beta");
    return SCCS_OK;
}

int sccs_check_wait_timeout(sccs_handle *h, double timeout_ms) {
    if (!h) return fail(SCCS_E_INVAL, "null handle");
    if (!(timeout_ms > 0.0 && timeout_ms <= 10000.0)) return fail(SCCS_E_INVAL, "timeout_ms must be in (0, 10000]");
    if (h->d.S < 2 || h->d.J < 1) return fail(SCCS_E_INVAL, "needs at least two shards and one column");
    int rc = set_device(h);
    if (rc) return rc;
    // One CTA fewer than the all-reduce expects: nothing ever writes the last slot, so every
    // launched CTA's bounded wait must run out and report the timeout.
    sccs::DevLayout d = h->d;
    d.S = h->d.S;  // the all-reduce still counts S participants
    sccs::FitParams p = base_params(h);
    p.timeout_ns = static_cast<long long>(timeout_ms * 1e6);
    cudaMemsetAsync(h->out_dev, 0, sizeof(sccs::FitOut), h->stream);
    int le = sccs::launch_grad_hess_partial(d, 0, p, h->out_dev, h->threads, h->d.S - 1, h->stream);
    if (le != 0) return cuda_fail(static_cast<cudaError_t>(le), "grad_hess kernel launch");
    if ((rc = sync_out(h))) return rc;
    const sccs::FitOut r = *h->out_host;
    reset_after_abort(h);
    if (r.status == -6 && r.abort_flag) return fail(SCCS_E_TIMEOUT, "bounded wait ran out as expected");
    return fail(SCCS_E_INVAL, "the wait did not time out");
}

}  // extern "C"
