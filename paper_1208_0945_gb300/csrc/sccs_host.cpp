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
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "sccs.h"
#include "sccs_internal.h"
#include "sccs_layout.h"

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

// Split [0, n) into `parts` contiguous chunks (the same cuts for the same n and parts) and run
// f(chunk, lo, hi) for each on the thread pool.
template <class F>
void parallel_chunks(int64_t n, int64_t parts, F f) {
    parts = std::max<int64_t>(1, parts);
    parallel_for(parts, [&](int64_t c) { f(c, n * c / parts, n * (c + 1) / parts); });
}

int64_t host_threads() {
    const unsigned hw = std::thread::hardware_concurrency();
    return hw ? static_cast<int64_t>(hw) : 4;
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
    // subject weights (Section 2.5): host maps, and device scratch made on first use
    std::vector<int64_t> kept_from;    // N: input subject of each kept subject
    std::vector<int32_t> nev_host;     // N: n_i
    int32_t max_nev = 0;
    int32_t *w_dev = nullptr;          // N: weights per kept subject
    int32_t *nev_w = nullptr;          // N: w_i n_i
    double *ytx_w = nullptr;           // J: weighted Y'X_j
    int32_t *w_host = nullptr;         // N, pinned
    bool e_stale = false;              // the FP64 E no longer matches beta (after an FP32-only fit)
    // the layout's arrays by SCCS_DBG_* id, for the layout diagnostic: address and size
    struct DbgArr {
        const void *p = nullptr;
        int64_t bytes = 0;
        bool host = false;
    };
    DbgArr dbg[SCCS_DBG_COUNT];
    std::vector<int64_t> cshard_row_h, cshard_pat_h, scalars_h;
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

// A new device array of `count` elements that a layout kernel fills; `pad` zeroed bytes follow
// (arrays read by bulk copies rounded out to 16-byte boundaries).
template <class T>
int alloc_padded(sccs_handle *h, T **dst, size_t count, size_t pad = 0) {
    *dst = static_cast<T *>(h->arena.get(count * sizeof(T) + pad));
    if (!*dst) return fail(SCCS_E_NOMEM, "device allocation failed");
    if (pad) {
        cudaError_t e = cudaMemsetAsync(reinterpret_cast<char *>(*dst) + count * sizeof(T), 0, pad, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    }
    return SCCS_OK;
}

// A new device array holding a copy of `count` elements of device memory.
template <class T>
int copy_in(sccs_handle *h, T **dst, const T *src, size_t count) {
    int rc = alloc_padded(h, dst, count);
    if (rc) return rc;
    if (count) {
        cudaError_t e = cudaMemcpyAsync(*dst, src, count * sizeof(T), cudaMemcpyDeviceToDevice, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync D2D");
    }
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
    if (h->w_host) cudaFreeHost(h->w_host);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

constexpr int32_t kNarrowDefault = 1024;
constexpr int32_t kClusterDefault = 16;
constexpr int64_t kClusterMaxNnzDefault = 8192;
using sccs::kNarrowGroupMax;
constexpr int32_t kNarrowMinShards = 4;

// Checks everything about the inputs that needs no GPU.
// The smallest i in [0, n) with bad(i), or -1: chunks in parallel, each stopping at its first.
template <class F>
int64_t first_bad(int64_t n, F bad) {
    if (n <= 0) return -1;
    const int64_t P = std::max<int64_t>(1, std::min<int64_t>(8 * host_threads(), n / 65536 + 1));
    std::vector<int64_t> f(static_cast<size_t>(P), -1);
    parallel_chunks(n, P, [&](int64_t c, int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; ++i)
            if (bad(i)) {
                f[c] = i;
                return;
            }
    });
    for (int64_t c = 0; c < P; ++c)
        if (f[c] >= 0) return f[c];
    return -1;
}

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
    int64_t k = first_bad(K - 1, [&](int64_t i) { return patient_id[i + 1] < patient_id[i]; });
    if (k >= 0) return fail(SCCS_E_UNSORTED, "patient_id decreases at row " + std::to_string(k + 1));
    k = first_bad(K, [&](int64_t i) { return y[i] < 0 || !(Lin[i] > 0.0) || !std::isfinite(Lin[i]); });
    if (k >= 0) {
        if (y[k] < 0) return fail(SCCS_E_INVAL, "negative event count at row " + std::to_string(k));
        return fail(SCCS_E_INVAL, "offset must be positive and finite at row " + std::to_string(k));
    }
    k = first_bad(nnz_in, [&](int64_t e) { return row_idx[e] < 0 || static_cast<int64_t>(row_idx[e]) >= K; });
    if (k >= 0) return fail(SCCS_E_INVAL, "row index out of range at nonzero " + std::to_string(k));
    if (x_values) {
        k = first_bad(nnz_in, [&](int64_t e) { return x_values[e] != 1.0; });
        if (k >= 0) return fail(SCCS_E_NONBINARY, "X value at nonzero " + std::to_string(k) + " is not 1");
    }
    // every n_i = 0: no subject contributes to Eq. 2, so there is nothing to fit
    if (first_bad(K, [&](int64_t i) { return y[i] > 0; }) < 0)
        return fail(SCCS_E_INVAL, "no events: every subject has n_i = 0");
    return SCCS_OK;
}

int run_init_state(sccs_handle *h, const double *beta_dev, bool keep_trust = false) {
    int e = sccs::launch_init_state(h->d, beta_dev, h->threads, h->stream, keep_trust);
    if (e != 0) return cuda_fail(static_cast<cudaError_t>(e), "init_state launch");
    h->e_stale = false;
    return SCCS_OK;
}

// Rebuild the FP64 state from the handle's own beta (trust radii kept) if an FP32-only fit
// left it behind.
int refresh_fp64_state(sccs_handle *h) {
    if (!h->e_stale) return SCCS_OK;
    cudaError_t e = cudaMemcpyAsync(h->beta_dev, h->d.beta_priv, sizeof(double) * std::max<int32_t>(h->d.J, 1),
                                    cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync beta");
    return run_init_state(h, h->beta_dev, true);
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

// Move the state to beta (host array) or keep the current one (nullptr; rebuilt in FP64 if an
// FP32-only fit left it behind).
int set_state(sccs_handle *h, const double *beta) {
    if (!beta) return refresh_fp64_state(h);
    const int32_t J = h->d.J;
    for (int32_t j = 0; j < J; ++j)
        if (!std::isfinite(beta[j])) return fail(SCCS_E_INVAL, "beta has a non-finite entry");
    std::memcpy(h->beta_host, beta, sizeof(double) * static_cast<size_t>(J));
    cudaError_t e = cudaMemcpyAsync(h->beta_dev, h->beta_host, sizeof(double) * std::max<int32_t>(J, 1),
                                    cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync beta");
    return run_init_state(h, h->beta_dev);
}

// E at the start of a cycle, for Genkin's X-beta convergence test (made on first use).
int ensure_e_prev(sccs_handle *h) {
    if (h->d.E_prev) return SCCS_OK;
    auto *p = static_cast<double *>(h->arena.get(sizeof(double) * static_cast<size_t>(std::max<int64_t>(h->d.K, 1))));
    if (!p) return fail(SCCS_E_NOMEM, "device memory for the X-beta test");
    h->d.E_prev = p;
    return SCCS_OK;
}

// ---- subject weights (Section 2.5)

int ensure_weight_scratch(sccs_handle *h) {
    if (h->w_dev) return SCCS_OK;
    const size_t N = static_cast<size_t>(std::max<int64_t>(h->d.N, 1));
    const size_t J = static_cast<size_t>(std::max<int32_t>(h->d.J, 1));
    auto *w = static_cast<int32_t *>(h->arena.get(4 * N));
    auto *nw = static_cast<int32_t *>(h->arena.get(4 * N));
    auto *yw = static_cast<double *>(h->arena.get(8 * J));
    if (!w || !nw || !yw) return fail(SCCS_E_NOMEM, "device memory for subject weights");
    if (cudaMallocHost(&h->w_host, 4 * N) != cudaSuccess) {
        (void)cudaGetLastError();
        h->w_host = nullptr;
        return fail(SCCS_E_NOMEM, "pinned memory for subject weights");
    }
    h->w_dev = w;
    h->nev_w = nw;
    h->ytx_w = yw;
    return SCCS_OK;
}

// Map the weights to kept subjects, upload them and form w_i n_i and the weighted Y'X_j.
int prepare_weights(sccs_handle *h, const int32_t *w_in) {
    int rc = ensure_weight_scratch(h);
    if (rc) return rc;
    sccs::HandleView v{};
    sccs_handle_view(h, &v);
    if ((rc = sccs::map_subject_weights(v, w_in, h->w_host))) return rc;
    cudaError_t e = cudaMemcpyAsync(h->w_dev, h->w_host, sizeof(int32_t) * static_cast<size_t>(std::max<int64_t>(h->d.N, 1)),
                                    cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync weights");
    const int le = sccs::launch_weighted_counts(h->d, h->w_dev, h->nev_w, h->ytx_w, h->stream);
    if (le != 0) return cuda_fail(static_cast<cudaError_t>(le), "weighted counts launch");
    return SCCS_OK;
}

// While alive, the handle's layout carries the weighted counts in place of n_i and Y'X_j.
struct CountsScope {
    sccs_handle *h;
    const int32_t *nev;
    const double *ytx;
    CountsScope(sccs_handle *hh, bool weighted) : h(hh), nev(hh->d.nev), ytx(hh->d.ytx) {
        if (weighted) {
            h->d.nev = h->nev_w;
            h->d.ytx = h->ytx_w;
        }
    }
    ~CountsScope() {
        h->d.nev = nev;
        h->d.ytx = ytx;
    }
};

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

// ------------------------------------------------------------------ batched fits
//
// A batch plan holds what one batch of handles needs on the device (entries, team offsets,
// counters, result buffers), pinned staging for the per-call entries and the results, and a
// CUDA graph of the whole device side of a call: entries in, counters and outputs zeroed, the
// persistent queue launch, the results gathered and copied out.  Plans are cached by handle
// list and precision and dropped when one of their handles is destroyed, so repeated batches
// over the same datasets (a prior-variance grid, say) replay the graph.
constexpr long long kAssembleWaitNs = 30000000000LL;   // a team waits at most 30 s for its CTAs
constexpr size_t kMaxPlans = 8;

struct BatchPlan {
    std::vector<sccs_handle *> handles;   // caller order
    int mode = 0;
    int device = 0;
    int n = 0;
    std::vector<int32_t> order;           // scheduling position -> caller index
    std::vector<long long> beta_off;      // per scheduling position, in doubles
    void *dev = nullptr;
    void *host = nullptr;
    size_t stage_bytes = 0, result_bytes = 0;
    sccs::BatchEntry *ent_host = nullptr;
    sccs::FitOut *out32_dev = nullptr;
    sccs::FitOut *res_outs_host = nullptr, *res_outs32_host = nullptr;
    double *res_beta_host = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long last_use = 0;
};

std::mutex g_batch_mu;
std::vector<BatchPlan *> g_plans;
unsigned long long g_plan_clock = 0;

void free_plan(BatchPlan *pl) {
    if (!pl) return;
    cudaSetDevice(pl->device);
    if (pl->stream) cudaStreamSynchronize(pl->stream);
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->dev) cudaFree(pl->dev);
    if (pl->host) cudaFreeHost(pl->host);
    if (pl->ev0) cudaEventDestroy(pl->ev0);
    if (pl->ev1) cudaEventDestroy(pl->ev1);
    if (pl->stream) cudaStreamDestroy(pl->stream);
    delete pl;
}

void forget_plans_of(const sccs_handle *h) {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (size_t i = 0; i < g_plans.size();) {
        BatchPlan *pl = g_plans[i];
        if (std::find(pl->handles.begin(), pl->handles.end(), h) != pl->handles.end()) {
            free_plan(pl);
            g_plans.erase(g_plans.begin() + static_cast<long>(i));
        } else {
            ++i;
        }
    }
}

size_t al256(size_t b) { return (b + 255) / 256 * 256; }

// Scheduling order: longest fits first (estimated device time per cycle: a latency term per
// coordinate plus the nonzeros and segments each CTA of the team streams).
std::vector<int32_t> lpt_order(sccs_handle *const *handles, int32_t n) {
    std::vector<double> cost(n);
    for (int32_t k = 0; k < n; ++k) {
        const sccs_handle *h = handles[k];
        cost[k] = 8192.0 * h->d.J +
                  (static_cast<double>(h->info.nnz_kept) + 2.0 * static_cast<double>(h->info.segments)) /
                      std::max(1, h->d.S);
    }
    std::vector<int32_t> order(n);
    for (int32_t k = 0; k < n; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
    return order;
}

// Called with g_batch_mu held.
int get_batch_plan(sccs_handle *const *handles, int32_t n, int mode, BatchPlan **out) {
    for (BatchPlan *pl : g_plans) {
        if (pl->mode == mode && pl->n == n && std::equal(pl->handles.begin(), pl->handles.end(), handles)) {
            pl->last_use = ++g_plan_clock;
            *out = pl;
            return SCCS_OK;
        }
    }
    const int threads = handles[0]->threads;
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, handles[0]->device);
    int rc = sccs::fit_kernel_max_blocks_per_sm(threads, &per_sm);
    if (rc) return cuda_fail(static_cast<cudaError_t>(rc), "occupancy");
    const int capacity = sms * std::max(per_sm, 1);
    long long tickets = 0;
    for (int32_t k = 0; k < n; ++k) {
        if (handles[k]->d.S > capacity) return fail(SCCS_E_INVAL, "a handle has more shards than the device holds at once");
        tickets += handles[k]->d.S;
    }
    auto pl = new BatchPlan();
    auto bail = [&](int code) {
        free_plan(pl);
        return code;
    };
    pl->handles.assign(handles, handles + n);
    pl->mode = mode;
    pl->device = handles[0]->device;
    pl->n = n;
    pl->order = lpt_order(handles, n);
    pl->beta_off.resize(n);
    long long nbeta = 0;
    std::vector<int> team_start(n + 1, 0);
    for (int32_t q = 0; q < n; ++q) {
        const sccs_handle *h = handles[pl->order[q]];
        pl->beta_off[q] = nbeta;
        nbeta += std::max<int32_t>(h->d.J, 1);
        team_start[q + 1] = team_start[q] + h->d.S;
    }
    // device: [entries | team_start | beta_off | counters | out32] [outs | outs32 | betas]
    const size_t b_ent = al256(sizeof(sccs::BatchEntry) * n), b_ts = al256(sizeof(int) * (n + 1)),
                 b_off = al256(sizeof(long long) * n), b_cnt = al256(sizeof(unsigned) * (n + 1)),
                 b_o32 = al256(sizeof(sccs::FitOut) * n), b_outs = al256(sizeof(sccs::FitOut) * n),
                 b_beta = al256(sizeof(double) * static_cast<size_t>(nbeta));
    pl->stage_bytes = b_ent + b_ts + b_off;
    pl->result_bytes = 2 * b_outs + b_beta;
    const size_t dev_bytes = pl->stage_bytes + b_cnt + b_o32 + pl->result_bytes;
    if (cudaMalloc(&pl->dev, dev_bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        pl->dev = nullptr;
        return bail(fail(SCCS_E_NOMEM, "batch buffers"));
    }
    if (cudaMallocHost(&pl->host, pl->stage_bytes + pl->result_bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        pl->host = nullptr;
        return bail(fail(SCCS_E_NOMEM, "batch staging"));
    }
    char *d = static_cast<char *>(pl->dev);
    char *hs = static_cast<char *>(pl->host);
    auto *ent_dev = reinterpret_cast<sccs::BatchEntry *>(d);
    auto *ts_dev = reinterpret_cast<int *>(d + b_ent);
    auto *off_dev = reinterpret_cast<long long *>(d + b_ent + b_ts);
    auto *cnt_dev = reinterpret_cast<unsigned *>(d + pl->stage_bytes);
    pl->out32_dev = reinterpret_cast<sccs::FitOut *>(d + pl->stage_bytes + b_cnt);
    char *res_dev = d + pl->stage_bytes + b_cnt + b_o32;
    auto *outs_dev = reinterpret_cast<sccs::FitOut *>(res_dev);
    auto *outs32_dev = reinterpret_cast<sccs::FitOut *>(res_dev + b_outs);
    auto *beta_dev = reinterpret_cast<double *>(res_dev + 2 * b_outs);
    pl->ent_host = reinterpret_cast<sccs::BatchEntry *>(hs);
    std::memcpy(hs + b_ent, team_start.data(), sizeof(int) * (n + 1));
    std::memcpy(hs + b_ent + b_ts, pl->beta_off.data(), sizeof(long long) * n);
    char *res_host = hs + pl->stage_bytes;
    pl->res_outs_host = reinterpret_cast<sccs::FitOut *>(res_host);
    pl->res_outs32_host = reinterpret_cast<sccs::FitOut *>(res_host + b_outs);
    pl->res_beta_host = reinterpret_cast<double *>(res_host + 2 * b_outs);
    if (cudaStreamCreateWithFlags(&pl->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&pl->ev0) != cudaSuccess || cudaEventCreate(&pl->ev1) != cudaSuccess) {
        (void)cudaGetLastError();
        return bail(fail(SCCS_E_CUDA, "batch stream or events"));
    }
    const int grid = static_cast<int>(std::min<long long>(tickets, capacity));
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(pl->stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return bail(cuda_fail(e, "batch capture"));
    int le = static_cast<int>(cudaMemcpyAsync(pl->dev, pl->host, pl->stage_bytes, cudaMemcpyHostToDevice, pl->stream));
    if (!le) le = sccs::launch_batch_prep(ent_dev, n, cnt_dev, pl->stream);
    if (!le) le = sccs::launch_fit_queue(ent_dev, ts_dev, n, cnt_dev, grid, threads, pl->stream, mode, kAssembleWaitNs);
    if (!le) le = sccs::launch_batch_gather(ent_dev, n, outs_dev, outs32_dev, beta_dev, off_dev, pl->stream);
    if (!le)
        le = static_cast<int>(cudaMemcpyAsync(res_host, res_dev, pl->result_bytes, cudaMemcpyDeviceToHost, pl->stream));
    e = cudaStreamEndCapture(pl->stream, &graph);
    if (le) {
        if (graph) cudaGraphDestroy(graph);
        (void)cudaGetLastError();
        return bail(cuda_fail(static_cast<cudaError_t>(le), "batch capture (launch)"));
    }
    if (e != cudaSuccess) return bail(cuda_fail(e, "batch capture (end)"));
    e = cudaGraphInstantiate(&pl->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        pl->exec = nullptr;
        return bail(cuda_fail(e, "batch graph instantiate"));
    }
    if (g_plans.size() >= kMaxPlans) {
        auto lru = std::min_element(g_plans.begin(), g_plans.end(),
                                    [](const BatchPlan *a, const BatchPlan *b) { return a->last_use < b->last_use; });
        free_plan(*lru);
        g_plans.erase(lru);
    }
    pl->last_use = ++g_plan_clock;
    g_plans.push_back(pl);
    *out = pl;
    return SCCS_OK;
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
    v->kept_from = h->kept_from.data();
    v->nev_host = h->nev_host.data();
    v->subjects_in = h->info.subjects_in;
    v->max_nev = h->max_nev;
    return true;
}

namespace sccs {

int map_subject_weights(const HandleView &v, const int32_t *w_in, int32_t *w_kept) {
    for (int64_t i = 0; i < v.d.N; ++i) {
        const int64_t src = v.kept_from[i];
        const int32_t w = w_in[src];
        if (w < 0) return fail(SCCS_E_INVAL, "negative weight for input subject " + std::to_string(src));
        if (static_cast<int64_t>(w) * v.nev_host[i] > INT32_MAX)
            return fail(SCCS_E_INVAL, "weight x events exceeds 2^31 - 1 for input subject " + std::to_string(src));
        w_kept[i] = w;
    }
    return SCCS_OK;
}

}  // namespace sccs

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
    // cluster columns: a cluster of C CTAs, and a team of whole clusters
    int32_t C = o.cluster_ctas < 0 ? 0 : (o.cluster_ctas == 0 ? (o.num_shards == 0 ? kClusterDefault : 0) : o.cluster_ctas);
    if (C != 0 && C != 2 && C != 4 && C != 8 && C != 16)
        return fail(SCCS_E_INVAL, "cluster_ctas must be 2, 4, 8 or 16 (0 = default, < 0 = off)");
    if (C > 0) {
        int ncl = 0;
        const int ce2 = sccs::fit_kernel_max_clusters(threads, C, &ncl);
        if (ce2 != 0 || ncl < 1) {
            if (o.cluster_ctas > 0) return fail(SCCS_E_UNSUPPORTED, "the device cannot hold clusters of that size");
            C = 0;   // the default quietly falls back to whole-team columns
        } else if (o.num_shards == 0) {
            S = std::min(S, ncl * C);
        } else if (S % C != 0 || S > ncl * C) {
            return fail(SCCS_E_INVAL, "with cluster_ctas, num_shards must be a multiple of it and at most " +
                                          std::to_string(ncl * C));
        }
    }
    const int64_t cluster_max = o.cluster_max_nnz > 0 ? o.cluster_max_nnz : kClusterMaxNnzDefault;

    const int32_t narrow_max = o.narrow_max_nnz == 0 ? kNarrowDefault : o.narrow_max_nnz;
    // every column of a group keeps at least two warps of the CTA
    const int32_t group_cap = std::max(1, std::min(kNarrowGroupMax, threads / 64));
    const int32_t group_max = o.narrow_group_max <= 0 ? group_cap : std::min(o.narrow_group_max, group_cap);
    // when every column small enough for the narrow path is a cluster column as well, the cluster
    // takes them all and no narrow layout is built
    const int32_t narrow_eff = (C > 0 && cluster_max >= narrow_max) ? -1 : narrow_max;

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
    // the layout's scratch (device) and the pinned words its stages read back
    sccs::lay::Scratch scr(h->stream);
    unsigned long long *pinned = nullptr;
    auto bail = [&](int code) {
        std::string msg = g_last_error;
        scr.release();
        if (h->stream) cudaStreamSynchronize(h->stream);
        if (pinned) cudaFreeHost(pinned);
        destroy_handle(h);
        g_last_error = msg;
        return code;
    };
    int rc = SCCS_OK;
    auto lay_fail = [&](int e, const char *what) { return bail(cuda_fail(static_cast<cudaError_t>(e), what)); };
    if ((ce = cudaEventCreate(&h->ev0)) != cudaSuccess || (ce = cudaEventCreate(&h->ev1)) != cudaSuccess)
        return bail(cuda_fail(ce, "cudaEventCreate"));
    if ((ce = cudaMallocHost(&h->out_host, sizeof(sccs::FitOut))) != cudaSuccess)
        return bail(cuda_fail(ce, "cudaMallocHost"));
    if ((ce = cudaMallocHost(&h->beta_host, sizeof(double) * std::max<int32_t>(J, 1))) != cudaSuccess)
        return bail(cuda_fail(ce, "cudaMallocHost"));
    if ((ce = cudaMallocHost(&pinned, sizeof(unsigned long long) * (sccs::lay::kFCount + 2))) != cudaSuccess)
        return bail(cuda_fail(ce, "cudaMallocHost"));

    // ---- the layout, on the device (sccs_layout.cu); the host decides over columns
    namespace lay = sccs::lay;
    lay::Ctx c;
    c.st = h->stream;
    c.scr = &scr;
    c.K = K;
    c.nnz_in = col_ptr[J];
    c.J = J;
    c.flags_h = pinned;
    c.total_h = reinterpret_cast<long long *>(pinned + lay::kFCount);
    int le = lay::upload_inputs(c, patient_id, y, offset_L, col_ptr, row_idx);
    if (le) return lay_fail(le, "layout: input upload");
    h->arena.uploaded += K * (8 + 4 + 8) + 8 * (static_cast<int64_t>(J) + 1) + 4 * c.nnz_in;
    // subjects, n_i, dropping n_i = 0
    if ((le = lay::subjects_count(c))) return lay_fail(le, "layout: subjects");
    if (c.Kk >= (int64_t(1) << 31)) return bail(fail(SCCS_E_INVAL, "more than 2^31-1 kept rows"));
    if (c.flags_h[lay::kFBigN]) return bail(fail(SCCS_E_INVAL, "n_i exceeds 2^31-1"));
    const int64_t Nk = c.Nk, Kk = c.Kk;
    int64_t *pat_s = scr.get_n<int64_t>(static_cast<size_t>(Nk) + 1);
    int32_t *nev_s = scr.get_n<int32_t>(static_cast<size_t>(Nk));
    int64_t *kf_s = scr.get_n<int64_t>(static_cast<size_t>(Nk));
    double *L_s = scr.get_n<double>(static_cast<size_t>(Kk));
    if (!pat_s || !nev_s || !kf_s || !L_s) return bail(fail(SCCS_E_NOMEM, "layout scratch"));
    if ((le = lay::subjects_fill(c, pat_s, nev_s, kf_s, L_s))) return lay_fail(le, "layout: subjects");
    // columns: kept rows ascending, duplicates, Y'X_j
    std::vector<int64_t> cptr, ytx_i, cseg;
    if ((le = lay::columns(c, cptr, ytx_i))) return lay_fail(le, "layout: columns");
    if (c.flags_h[lay::kFDup] != lay::kNone)
        return bail(fail(SCCS_E_DUPLICATE, "a row appears twice in column " + std::to_string(c.flags_h[lay::kFDup])));
    if ((le = lay::segments(c, cseg))) return lay_fail(le, "layout: segments");
    lay::ScanBuf pair_sb;
    int64_t npairs = 0;
    if ((le = lay::pairs_count(c, pair_sb, npairs))) return lay_fail(le, "layout: pairs");
    // shards at subject boundaries, balanced by rows, and their slices
    int64_t *shard_pat_s = scr.get_n<int64_t>(static_cast<size_t>(S) + 1);
    int64_t *shard_row_s = scr.get_n<int64_t>(static_cast<size_t>(S) + 1);
    if (!shard_pat_s || !shard_row_s) return bail(fail(SCCS_E_NOMEM, "layout scratch"));
    if ((le = lay::shards(c, pat_s, S, shard_pat_s, shard_row_s))) return lay_fail(le, "layout: shards");
    lay::SliceSet ss;
    ss.Sp = S;
    ss.shard_pat = shard_pat_s;
    if ((le = lay::slices_count(c, ss, nullptr, nullptr))) return lay_fail(le, "layout: slices");
    int64_t max_col = 0;
    for (int32_t j = 0; j < J; ++j) max_col = std::max<int64_t>(max_col, cptr[j + 1] - cptr[j]);

    sccs::DevLayout &d = h->d;
    d.S = S;
    d.J = J;
    d.K = Kk;
    d.N = Nk;
    const size_t SJ = static_cast<size_t>(S) * (static_cast<size_t>(J) + 1);
    int32_t *rows;
    int2 *segs;
    int64_t *grp_base, *slice_row, *slice_seg, *slice_grp, *shard_row, *shard_pat, *pat_ptr;
    int32_t *nev, *ysub, *ycnt;
    double *L, *ytx;
    int64_t *ycol_ptr;
    std::vector<double> ytx_h(static_cast<size_t>(J));
    for (int32_t j = 0; j < J; ++j) ytx_h[j] = static_cast<double>(ytx_i[j]);   // exact below 2^53
    // allocation order as measured fastest for the fit: static structure, then the state
    if ((rc = alloc_padded(h, &rows, static_cast<size_t>(ss.tr), sccs::kCopyPad)) ||
        (rc = alloc_padded(h, &segs, static_cast<size_t>(ss.ts), sccs::kCopyPad)) ||
        (rc = alloc_padded(h, &grp_base, static_cast<size_t>(ss.tg), sccs::kCopyPad)) ||
        (rc = alloc_padded(h, &slice_row, SJ)) || (rc = alloc_padded(h, &slice_seg, SJ)) ||
        (rc = alloc_padded(h, &slice_grp, SJ)) ||
        (rc = copy_in(h, &shard_row, shard_row_s, static_cast<size_t>(S) + 1)) ||
        (rc = copy_in(h, &shard_pat, shard_pat_s, static_cast<size_t>(S) + 1)) ||
        (rc = copy_in(h, &pat_ptr, pat_s, static_cast<size_t>(Nk) + 1)) ||
        (rc = copy_in(h, &nev, nev_s, static_cast<size_t>(Nk))) || (rc = copy_in(h, &L, L_s, static_cast<size_t>(Kk))) ||
        (rc = upload(h, &ytx, ytx_h.data(), ytx_h.size())))
        return bail(rc);
    if ((le = lay::slices_fill(c, ss, slice_row, slice_seg, slice_grp, rows, segs, grp_base)))
        return lay_fail(le, "layout: slices");
    auto reg = [&](int id, const void *p, int64_t bytes, bool host = false) { h->dbg[id] = {p, bytes, host}; };
    reg(SCCS_DBG_ROWS, rows, 4 * ss.tr);
    reg(SCCS_DBG_SEGS, segs, 8 * ss.ts);
    reg(SCCS_DBG_GRP_BASE, grp_base, 8 * ss.tg);
    reg(SCCS_DBG_SLICE_ROW, slice_row, 8 * static_cast<int64_t>(SJ));
    reg(SCCS_DBG_SLICE_SEG, slice_seg, 8 * static_cast<int64_t>(SJ));
    reg(SCCS_DBG_SLICE_GRP, slice_grp, 8 * static_cast<int64_t>(SJ));
    reg(SCCS_DBG_SHARD_ROW, shard_row, 8 * (static_cast<int64_t>(S) + 1));
    reg(SCCS_DBG_SHARD_PAT, shard_pat, 8 * (static_cast<int64_t>(S) + 1));
    reg(SCCS_DBG_PAT_PTR, pat_ptr, 8 * (Nk + 1));
    reg(SCCS_DBG_NEV, nev, 4 * Nk);
    reg(SCCS_DBG_L, L, 8 * Kk);
    reg(SCCS_DBG_YTX, ytx, 8 * static_cast<int64_t>(J));
    h->kept_from.resize(static_cast<size_t>(Nk));
    h->nev_host.resize(static_cast<size_t>(Nk));
    if (Nk > 0) {
        if ((ce = cudaMemcpyAsync(h->kept_from.data(), kf_s, 8 * static_cast<size_t>(Nk), cudaMemcpyDeviceToHost,
                                  h->stream)) != cudaSuccess ||
            (ce = cudaMemcpyAsync(h->nev_host.data(), nev_s, 4 * static_cast<size_t>(Nk), cudaMemcpyDeviceToHost,
                                  h->stream)) != cudaSuccess)
            return bail(cuda_fail(ce, "cudaMemcpyAsync D2H"));
    }
    for (int32_t v : h->nev_host) h->max_nev = std::max(h->max_nev, v);
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
    d.stash_stride = ss.max_seg;
    if ((rc = alloc_zero(h, &d.E, static_cast<size_t>(Kk))) ||
        (rc = alloc_zero(h, &d.D, static_cast<size_t>(Nk))) ||
        (rc = alloc_zero(h, &d.E32, static_cast<size_t>(Kk))) ||
        (rc = alloc_zero(h, &d.D32, static_cast<size_t>(Nk))) ||
        (rc = alloc_zero(h, &d.beta_priv, static_cast<size_t>(S) * std::max<int32_t>(J, 1))) ||
        (rc = alloc_zero(h, &d.trust_priv, static_cast<size_t>(S) * std::max<int32_t>(J, 1))) ||
        (rc = alloc_zero(h, &d.stash, static_cast<size_t>(S) * 2 * static_cast<size_t>(ss.max_seg))) ||
        (rc = alloc_zero(h, &d.slots, static_cast<size_t>(S) * 4)) ||
        (rc = alloc_zero(h, &h->out_dev, 1)) ||
        (rc = alloc_zero(h, &h->beta_dev, static_cast<size_t>(std::max<int32_t>(J, 1)))))
        return bail(rc);
    d.abort_flag = &h->out_dev->abort_flag;
    // The weighted-count pairs go last: the fit's state arrays keep the placement measured
    // fastest (placing 2 x 16 MB of pairs before them cost the 1M-subject fit 4%).
    std::vector<int64_t> ycol_h;
    if ((rc = alloc_padded(h, &ycol_ptr, static_cast<size_t>(J) + 1)) ||
        (rc = alloc_padded(h, &ysub, static_cast<size_t>(npairs))) ||
        (rc = alloc_padded(h, &ycnt, static_cast<size_t>(npairs))))
        return bail(rc);
    if ((le = lay::pairs_fill(c, pair_sb, npairs, ysub, ycnt, ycol_h))) return lay_fail(le, "layout: pairs");
    if ((ce = cudaMemcpyAsync(ycol_ptr, ycol_h.data(), 8 * ycol_h.size(), cudaMemcpyHostToDevice, h->stream)) !=
        cudaSuccess)
        return bail(cuda_fail(ce, "cudaMemcpyAsync H2D"));
    d.ycol_ptr = ycol_ptr;
    d.ysub = ysub;
    d.ycnt = ycnt;
    reg(SCCS_DBG_YCOL_PTR, ycol_ptr, 8 * (static_cast<int64_t>(J) + 1));
    reg(SCCS_DBG_YSUB, ysub, 4 * npairs);
    reg(SCCS_DBG_YCNT, ycnt, 4 * npairs);
    {
        // row -> columns index, built on the device from the slices (scratch freed with the rest)
        int64_t *row_ptr = nullptr;
        int32_t *row_col = nullptr;
        if ((rc = alloc_zero(h, &row_ptr, static_cast<size_t>(Kk) + 1)) ||
            (rc = alloc_zero(h, &row_col, static_cast<size_t>(c.nnz))))
            return bail(rc);
        const size_t K1 = static_cast<size_t>(std::max<int64_t>(Kk, 1));
        int32_t *cnt = scr.get_n<int32_t>(K1);
        int64_t *cursor = scr.get_n<int64_t>(K1);
        int64_t *sums = scr.get_n<int64_t>(sccs::row_index_scan_blocks(Kk));
        if (!cnt || !cursor || !sums) return bail(fail(SCCS_E_NOMEM, "row index scratch"));
        if ((le = sccs::launch_build_row_index(d, row_ptr, row_col, cnt, cursor, sums, h->stream)))
            return lay_fail(le, "row index build");
        d.row_ptr = row_ptr;
        d.row_col = row_col;
        reg(SCCS_DBG_ROW_PTR, row_ptr, 8 * (Kk + 1));
        reg(SCCS_DBG_ROW_COL, row_col, 4 * c.nnz);
    }
    std::vector<int32_t> nseg_col(static_cast<size_t>(J));
    for (int32_t j = 0; j < J; ++j) nseg_col[j] = static_cast<int32_t>(cseg[j + 1] - cseg[j]);
    // ---- narrow columns: few rows and subjects, run whole on one CTA
    int32_t narrow_count = 0, first_wide_col = -1;
    if (narrow_eff > 0 && S >= kNarrowMinShards) {
        std::vector<uint8_t> narrow(static_cast<size_t>(J), 0);
        std::vector<int64_t> nar_ptr(static_cast<size_t>(J) + 1, 0), row_first(static_cast<size_t>(J), 0);
        int64_t rows_total = 0;
        std::vector<int32_t> ncols;
        for (int32_t j = 0; j < J; ++j) {
            const int64_t n = cptr[j + 1] - cptr[j];
            // half the shared buffers each: the next column is gathered while this one steps
            const bool fits = n <= narrow_eff && n <= sccs::kRowCap / 2 && nseg_col[j] <= sccs::kSegCap / 2 &&
                              rows_total + n < (int64_t(1) << 31);
            narrow[j] = fits ? 1 : 0;
            nar_ptr[j + 1] = nar_ptr[j] + (fits ? nseg_col[j] : 0);
            row_first[j] = rows_total;
            if (fits) {
                rows_total += n;
                ncols.push_back(j);
            }
        }
        narrow_count = static_cast<int32_t>(ncols.size());
        if (narrow_count > 0) {
            std::vector<int32_t> lp_n;
            if ((le = lay::last_prev_columns(c, pat_ptr, d.row_ptr, d.row_col, ncols, lp_n)))
                return lay_fail(le, "layout: narrow groups");
            std::vector<int32_t> lp(static_cast<size_t>(J), -1);
            for (size_t q = 0; q < ncols.size(); ++q) lp[ncols[q]] = lp_n[q];
            // Groups: consecutive narrow columns with pairwise disjoint subjects (no column of the
            // group before jn shares a subject with jn: lp[jn] < j).  Neither column of a pair
            // reads what the other writes (their subjects' E and D), so their coordinate steps
            // can be taken side by side and give exactly the sequential result.  A group fits
            // half the shared buffers (rows, segments), like one narrow column.
            std::vector<int32_t> nar_group(static_cast<size_t>(J), 0);
            for (int32_t j = 0; j < J;) {
                if (!narrow[j]) {
                    ++j;
                    continue;
                }
                int32_t m = 1;
                int64_t sg = nseg_col[j], rw = cptr[j + 1] - cptr[j];
                while (j + m < J && narrow[j + m] && m < group_max) {
                    const int32_t jn = j + m;
                    if (sg + nseg_col[jn] > sccs::kSegCap / 2 || rw + (cptr[jn + 1] - cptr[jn]) > sccs::kRowCap / 2)
                        break;
                    if (lp[jn] >= j) break;
                    sg += nseg_col[jn];
                    rw += cptr[jn + 1] - cptr[jn];
                    ++m;
                }
                nar_group[j] = m;
                j += m;
            }
            // A group's state is gathered before the step ahead of it has written E and D: the
            // run's first group while the wide column before the run is still being applied on
            // the other shards, a later group while the previous group steps.  Each segment
            // records the one step that can change its subject: w = c + 1 if the subject is in
            // column c of the previous group, kNarrowAfterWide if the run's preceding wide column
            // touches it, else 0.  The kernel gathers a segment again when that step was not zero.
            std::vector<lay::NarrowCol> meta;
            meta.reserve(ncols.size());
            int32_t prev0 = -1, prevm = 0;
            for (int32_t g = 0; g < J;) {
                if (!narrow[g]) {
                    ++g;
                    continue;
                }
                const int32_t m = nar_group[g];
                const bool run_start = g == 0 || !narrow[g - 1];
                for (int32_t q = g; q < g + m; ++q) {
                    lay::NarrowCol nc{};
                    nc.j = q;
                    nc.run_wide = run_start && g > 0 ? g - 1 : -1;
                    nc.prev0 = run_start ? -1 : prev0;
                    nc.prevm = run_start ? 0 : prevm;
                    nc.nar_first = nar_ptr[q];
                    nc.row_first = row_first[q];
                    meta.push_back(nc);
                }
                prev0 = g;
                prevm = m;
                g += m;
            }
            std::vector<int32_t> next_wide(static_cast<size_t>(J), 0);
            int32_t first_wide = -1;
            for (int32_t j = 0; j < J; ++j)
                if (!narrow[j]) {
                    first_wide = j;
                    break;
                }
            {
                int32_t nxt = first_wide;
                for (int32_t j = J - 1; j >= 0; --j) {
                    next_wide[j] = nxt;
                    if (!narrow[j]) nxt = j;
                }
            }
            uint8_t *nar;
            int32_t *nxt, *nrow, *ngrp;
            int64_t *nptr;
            int4 *nseg;
            unsigned long long *nsync;
            if ((rc = upload(h, &nar, narrow.data(), narrow.size())) ||
                (rc = upload(h, &nxt, next_wide.data(), next_wide.size())) ||
                (rc = upload(h, &nptr, nar_ptr.data(), nar_ptr.size())) ||
                (rc = alloc_padded(h, &nseg, static_cast<size_t>(nar_ptr[J]))) ||
                (rc = alloc_padded(h, &nrow, static_cast<size_t>(rows_total))) ||
                (rc = upload(h, &ngrp, nar_group.data(), nar_group.size())) ||
                (rc = alloc_zero(h, &nsync, static_cast<size_t>(32))))
                return bail(rc);
            if ((le = lay::narrow_fill(c, pat_ptr, d.row_ptr, d.row_col, meta, nseg, nrow, sccs::kNarrowAfterWide)))
                return lay_fail(le, "layout: narrow columns");
            d.narrow = nar;
            d.next_wide = nxt;
            d.first_wide = first_wide;
            first_wide_col = first_wide;
            reg(SCCS_DBG_NARROW, nar, J);
            reg(SCCS_DBG_NEXT_WIDE, nxt, 4 * static_cast<int64_t>(J));
            reg(SCCS_DBG_NAR_PTR, nptr, 8 * (static_cast<int64_t>(J) + 1));
            reg(SCCS_DBG_NAR_SEG, nseg, 16 * nar_ptr[J]);
            reg(SCCS_DBG_NAR_ROW, nrow, 4 * rows_total);
            reg(SCCS_DBG_NAR_GROUP, ngrp, 4 * static_cast<int64_t>(J));
            d.nar_ptr = nptr;
            d.nar_seg = nseg;
            d.nar_row = nrow;
            d.nar_group = ngrp;
            d.nar_sync = nsync;
        }
    }
    // ---- cluster columns: at most cluster_max nonzeros, over C subject shards of their own, each
    //      slice small enough to be staged whole (else the column stays with the whole team)
    int32_t cluster_count = 0, first_grid_col = -1;
    if (C > 0) {
        int64_t *csp = scr.get_n<int64_t>(static_cast<size_t>(C) + 1);
        int64_t *csr_s = scr.get_n<int64_t>(static_cast<size_t>(C) + 1);
        uint8_t *mask_d = scr.get_n<uint8_t>(static_cast<size_t>(std::max<int32_t>(J, 1)));
        if (!csp || !csr_s || !mask_d) return bail(fail(SCCS_E_NOMEM, "layout scratch"));
        if ((le = lay::shards(c, pat_ptr, C, csp, csr_s))) return lay_fail(le, "layout: cluster shards");
        std::vector<uint8_t> ccls(static_cast<size_t>(J), 0);
        for (int32_t j = 0; j < J; ++j) ccls[j] = (cptr[j + 1] - cptr[j]) <= cluster_max ? 1 : 0;
        if (J > 0 && (ce = cudaMemcpyAsync(mask_d, ccls.data(), ccls.size(), cudaMemcpyHostToDevice, h->stream)) !=
                         cudaSuccess)
            return bail(cuda_fail(ce, "cudaMemcpyAsync H2D"));
        std::vector<int64_t> cnz, cns;
        lay::SliceSet cs;
        cs.Sp = C;
        cs.shard_pat = csp;
        cs.mask = mask_d;
        if ((le = lay::slices_count(c, cs, &cnz, &cns))) return lay_fail(le, "layout: cluster slices");
        auto at = [&](int32_t q, int32_t j) { return static_cast<size_t>(q) * (static_cast<size_t>(J) + 1) + j; };
        bool changed = false;
        for (int32_t j = 0; j < J; ++j) {
            if (!ccls[j]) continue;
            for (int32_t q = 0; q < C; ++q)
                if (cnz[at(q, j)] > sccs::kRowCap || cns[at(q, j)] > sccs::kSegCap) {
                    ccls[j] = 0;
                    changed = true;
                    break;
                }
        }
        if (changed) {
            if ((ce = cudaMemcpyAsync(mask_d, ccls.data(), ccls.size(), cudaMemcpyHostToDevice, h->stream)) !=
                cudaSuccess)
                return bail(cuda_fail(ce, "cudaMemcpyAsync H2D"));
            lay::SliceSet cs2;
            cs2.Sp = C;
            cs2.shard_pat = csp;
            cs2.mask = mask_d;
            cs = cs2;
            if ((le = lay::slices_count(c, cs, nullptr, nullptr))) return lay_fail(le, "layout: cluster slices");
        }
        std::vector<int32_t> ccols;
        for (int32_t j = 0; j < J; ++j)
            if (ccls[j]) ccols.push_back(j);
        cluster_count = static_cast<int32_t>(ccols.size());
        std::vector<int32_t> lp_c;
        if ((le = lay::last_prev_columns(c, pat_ptr, d.row_ptr, d.row_col, ccols, lp_c)))
            return lay_fail(le, "layout: cluster groups");
        std::vector<int32_t> lp(static_cast<size_t>(J), -1);
        for (size_t q = 0; q < ccols.size(); ++q) lp[ccols[q]] = lp_c[q];
        // Groups: consecutive cluster columns with pairwise disjoint subjects, up to group_max,
        // whose slices on every cluster shard fit one staging buffer together, formed greedily.
        // Neither column of a pair reads what the other writes, so their steps can be taken side
        // by side with exactly the sequential result.
        std::vector<int32_t> cgroup(static_cast<size_t>(J), 0);
        std::vector<int64_t> rows_c(static_cast<size_t>(C)), segs_c(static_cast<size_t>(C));
        for (int32_t j = 0; j < J;) {
            if (!ccls[j]) {
                ++j;
                continue;
            }
            for (int32_t q = 0; q < C; ++q) {
                rows_c[q] = cnz[at(q, j)];
                segs_c[q] = cns[at(q, j)];
            }
            int32_t m = 1;
            while (j + m < J && ccls[j + m] && m < group_max) {
                const int32_t jn = j + m;
                bool fits = lp[jn] < j;
                for (int32_t q = 0; q < C && fits; ++q)
                    fits = rows_c[q] + cnz[at(q, jn)] <= sccs::kRowCap && segs_c[q] + cns[at(q, jn)] <= sccs::kSegCap;
                if (!fits) break;
                for (int32_t q = 0; q < C; ++q) {
                    rows_c[q] += cnz[at(q, jn)];
                    segs_c[q] += cns[at(q, jn)];
                }
                ++m;
            }
            cgroup[j] = m;
            j += m;
        }
        int32_t first_grid = -1;
        for (int32_t j = 0; j < J; ++j)
            if (!ccls[j]) {
                first_grid = j;
                break;
            }
        std::vector<int32_t> next_grid(static_cast<size_t>(J), 0);
        {
            int32_t nxt = first_grid;
            for (int32_t j = J - 1; j >= 0; --j) {
                next_grid[j] = nxt;
                if (!ccls[j]) nxt = j;
            }
        }
        const size_t CJ = static_cast<size_t>(C) * (static_cast<size_t>(J) + 1);
        uint8_t *ccls_d;
        int32_t *ngrid, *crows, *cgrp_n;
        int2 *csegs;
        int64_t *cgrp, *csr, *css, *csg;
        unsigned long long *csync;
        if ((rc = upload(h, &ccls_d, ccls.data(), ccls.size())) ||
            (rc = upload(h, &ngrid, next_grid.data(), next_grid.size())) ||
            (rc = upload(h, &cgrp_n, cgroup.data(), cgroup.size())) ||
            (rc = alloc_padded(h, &crows, static_cast<size_t>(cs.tr), sccs::kCopyPad)) ||
            (rc = alloc_padded(h, &csegs, static_cast<size_t>(cs.ts), sccs::kCopyPad)) ||
            (rc = alloc_padded(h, &cgrp, static_cast<size_t>(cs.tg), sccs::kCopyPad)) ||
            (rc = alloc_padded(h, &csr, CJ)) || (rc = alloc_padded(h, &css, CJ)) || (rc = alloc_padded(h, &csg, CJ)) ||
            (rc = alloc_zero(h, &csync, static_cast<size_t>(32))))
            return bail(rc);
        if ((le = lay::slices_fill(c, cs, csr, css, csg, crows, csegs, cgrp)))
            return lay_fail(le, "layout: cluster slices");
        d.C = C;
        d.first_grid = first_grid;
        first_grid_col = first_grid;
        h->cshard_row_h.assign(static_cast<size_t>(C) + 1, 0);
        h->cshard_pat_h.assign(static_cast<size_t>(C) + 1, 0);
        if ((ce = cudaMemcpyAsync(h->cshard_row_h.data(), csr_s, 8 * (static_cast<size_t>(C) + 1),
                                  cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess ||
            (ce = cudaMemcpyAsync(h->cshard_pat_h.data(), csp, 8 * (static_cast<size_t>(C) + 1),
                                  cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess)
            return bail(cuda_fail(ce, "cudaMemcpyAsync D2H"));
        reg(SCCS_DBG_CCLS, ccls_d, J);
        reg(SCCS_DBG_NEXT_GRID, ngrid, 4 * static_cast<int64_t>(J));
        reg(SCCS_DBG_CGROUP, cgrp_n, 4 * static_cast<int64_t>(J));
        reg(SCCS_DBG_CROWS, crows, 4 * cs.tr);
        reg(SCCS_DBG_CSEGS, csegs, 8 * cs.ts);
        reg(SCCS_DBG_CGRP_BASE, cgrp, 8 * cs.tg);
        reg(SCCS_DBG_CSLICE_ROW, csr, 8 * static_cast<int64_t>(CJ));
        reg(SCCS_DBG_CSLICE_SEG, css, 8 * static_cast<int64_t>(CJ));
        reg(SCCS_DBG_CSLICE_GRP, csg, 8 * static_cast<int64_t>(CJ));
        reg(SCCS_DBG_CSHARD_ROW, h->cshard_row_h.data(), 8 * (static_cast<int64_t>(C) + 1), true);
        reg(SCCS_DBG_CSHARD_PAT, h->cshard_pat_h.data(), 8 * (static_cast<int64_t>(C) + 1), true);
        d.ccls = ccls_d;
        d.next_grid = ngrid;
        d.cgroup = cgrp_n;
        d.crows = crows;
        d.csegs = csegs;
        d.cgrp_base = cgrp;
        d.cslice_row = csr;
        d.cslice_seg = css;
        d.cslice_grp = csg;
        d.clu_sync = csync;
    }
    {
        // E per row of an unstaged slice between its phases A and C (allocated last: the arrays
        // above keep their measured placement)
        double *estash = nullptr;
        if ((rc = alloc_zero(h, &estash, static_cast<size_t>(S) * static_cast<size_t>(ss.max_rows))))
            return bail(rc);
        d.estash = estash;
        d.estash_stride = ss.max_rows;
    }
    if ((rc = run_init_state(h, nullptr))) return bail(rc);
    scr.release();
    ce = cudaStreamSynchronize(h->stream);
    if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaStreamSynchronize"));
    cudaFreeHost(pinned);
    pinned = nullptr;

    h->scalars_h = {c.nnz, c.nsub, narrow_count, cluster_count, first_grid_col, ss.max_seg, ss.max_rows,
                    first_wide_col};
    h->dbg[SCCS_DBG_SCALARS] = {h->scalars_h.data(), 8 * static_cast<int64_t>(h->scalars_h.size()), true};
    h->dbg[SCCS_DBG_KEPT_FROM] = {h->kept_from.data(), 8 * static_cast<int64_t>(h->kept_from.size()), true};
    sccs_data_info &info = h->info;
    info.rows_in = K;
    info.rows_kept = Kk;
    info.subjects_in = c.nsub;
    info.subjects_kept = Nk;
    info.nnz_kept = c.nnz;
    info.segments = ss.ts;
    info.max_column_nnz = max_col;
    info.device_bytes = h->arena.total;
    info.upload_bytes = h->arena.uploaded;
    info.columns = J;
    info.num_shards = S;
    info.threads_per_block = threads;
    info.narrow_columns = narrow_count;
    info.cluster_ctas = C;
    info.cluster_columns = cluster_count;
    *out = h;
    return SCCS_OK;
}

int sccs_debug_layout(const sccs_handle *h, int32_t which, void *dst, int64_t capacity, int64_t *bytes) {
    if (!h || !bytes) return fail(SCCS_E_INVAL, "null argument");
    if (which < 1 || which >= SCCS_DBG_COUNT) return fail(SCCS_E_INVAL, "unknown layout array");
    const sccs_handle::DbgArr &a = h->dbg[which];
    *bytes = a.p ? a.bytes : 0;
    if (!dst || *bytes == 0) return SCCS_OK;
    if (capacity < *bytes) return fail(SCCS_E_INVAL, "buffer too small for the layout array");
    if (a.host) {
        std::memcpy(dst, a.p, static_cast<size_t>(a.bytes));
        return SCCS_OK;
    }
    int rc = set_device(h);
    if (rc) return rc;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) e = cudaMemcpy(dst, a.p, static_cast<size_t>(a.bytes), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "layout copy");
    return SCCS_OK;
}

int sccs_destroy(sccs_handle *h) {
    if (h) forget_plans_of(h);
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
    if (o.tol_mode != SCCS_TOL_ABS_LOGPOST && o.tol_mode != SCCS_TOL_REL_LOGPOST &&
        o.tol_mode != SCCS_TOL_GENKIN_XBETA)
        return fail(SCCS_E_INVAL, "unknown tol_mode");
    if (o.precision != SCCS_PREC_FP64 && o.precision != SCCS_PREC_FP32_POLISH && o.precision != SCCS_PREC_FP32)
        return fail(SCCS_E_INVAL, "unknown precision");
    if (o.tol_mode == SCCS_TOL_GENKIN_XBETA && o.precision == SCCS_PREC_FP32)
        return fail(SCCS_E_UNSUPPORTED, "the Genkin X-beta test needs the FP64 state (use FP64 or FP32 + polish)");
    int rc = set_device(h);
    if (rc) return rc;
    if (o.tol_mode == SCCS_TOL_GENKIN_XBETA && (rc = ensure_e_prev(h))) return rc;
    if (o.subject_weights && (rc = prepare_weights(h, o.subject_weights))) return rc;
    CountsScope counts(h, o.subject_weights != nullptr);

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
    h->e_stale = o.precision == SCCS_PREC_FP32;   // the FP32 phase kept E in FP32 only
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
    if (o.tol_mode != SCCS_TOL_ABS_LOGPOST && o.tol_mode != SCCS_TOL_REL_LOGPOST &&
        o.tol_mode != SCCS_TOL_GENKIN_XBETA)
        return fail(SCCS_E_INVAL, "unknown tol_mode");
    if (o.precision != SCCS_PREC_FP64 && o.precision != SCCS_PREC_FP32_POLISH && o.precision != SCCS_PREC_FP32)
        return fail(SCCS_E_INVAL, "unknown precision");
    if (o.tol_mode == SCCS_TOL_GENKIN_XBETA && o.precision == SCCS_PREC_FP32)
        return fail(SCCS_E_UNSUPPORTED, "the Genkin X-beta test needs the FP64 state (use FP64 or FP32 + polish)");
    for (int32_t k = 0; k < n; ++k) {
        if (!handles[k]) return fail(SCCS_E_INVAL, "null handle in batch");
        if (handles[k]->device != handles[0]->device) return fail(SCCS_E_INVAL, "handles on different devices");
        if (handles[k]->threads != handles[0]->threads) return fail(SCCS_E_INVAL, "handles with different threads_per_block");
    }
    {
        std::vector<sccs_handle *> sorted(handles, handles + n);
        std::sort(sorted.begin(), sorted.end());
        if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
            return fail(SCCS_E_INVAL, "a handle appears twice in the batch");
    }
    sccs_handle *h0 = handles[0];
    int rc = set_device(h0);
    if (rc) return rc;
    const int mode = o.precision == SCCS_PREC_FP64 ? sccs::kBatchFp64
                     : o.precision == SCCS_PREC_FP32 ? sccs::kBatchFp32 : sccs::kBatchFp32Polish;
    if (o.tol_mode == SCCS_TOL_GENKIN_XBETA)
        for (int32_t k = 0; k < n; ++k)
            if ((rc = ensure_e_prev(handles[k]))) return rc;
    std::lock_guard<std::mutex> batch_lock(g_batch_mu);
    BatchPlan *plan = nullptr;
    if ((rc = get_batch_plan(handles, n, mode, &plan))) return rc;
    for (int32_t k = 0; k < n; ++k) {
        sccs_handle *h = handles[k];
        cudaError_t e = cudaStreamSynchronize(h->stream);   // no work of the handle in flight
        if (e != cudaSuccess) return cuda_fail(e, "handle stream");
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
    }
    // the entries, in the plan's scheduling order
    for (int32_t q = 0; q < n; ++q) {
        const int32_t k = plan->order[q];
        sccs_handle *h = handles[k];
        sccs::FitParams p = base_params(h);
        p.tol_mode = o.tol_mode;
        p.tol = o.tol;
        p.max_cycles = o.max_cycles;
        p.record_history = 1;
        sccs::FitParams p32 = p;
        if (mode == sccs::kBatchFp32Polish) {
            p32.tol_mode = SCCS_TOL_REL_LOGPOST;
            p32.tol = kFp32PhaseRelTol;
        }
        sccs::BatchEntry &en = plan->ent_host[q];
        en.d = h->d;
        en.p = p;
        en.p32 = p32;
        en.out = h->out_dev;
        en.out32 = mode == sccs::kBatchFp32Polish ? plan->out32_dev + q : nullptr;
        en.hist = h->hist_dev;
        en.warm = o.warm_start ? 1 : 0;
        en.team = h->d.S;
    }
    cudaEventRecord(plan->ev0, plan->stream);
    cudaError_t e = cudaGraphLaunch(plan->exec, plan->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch graph launch");
    cudaEventRecord(plan->ev1, plan->stream);
    e = cudaStreamSynchronize(plan->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch graph");
    float kms = 0.f;
    cudaEventElapsedTime(&kms, plan->ev0, plan->ev1);

    int first_err = SCCS_OK;
    for (int32_t q = 0; q < n; ++q) {
        const int32_t k = plan->order[q];
        sccs_handle *h = handles[k];
        const sccs::FitOut r = plan->res_outs_host[q];
        const sccs::FitOut r32 = mode == sccs::kBatchFp32Polish ? plan->res_outs32_host[q] : sccs::FitOut{};
        int status = SCCS_OK;
        if (r.status == -6 || r.abort_flag || r32.status == -6) {
            reset_after_abort(h);
            status = SCCS_E_TIMEOUT;
        } else if (r.status == -7 || r32.status == -7) {
            h->seq = r.status == -7 ? r.seq_end : r32.seq_end;
            run_init_state(h, nullptr);
            cudaStreamSynchronize(h->stream);
            status = SCCS_E_NUMERIC;
        } else {
            h->seq = r.seq_end;
            h->e_stale = mode == sccs::kBatchFp32;   // the FP32 phase kept E in FP32 only
        }
        const int32_t fp32_cycles = mode == sccs::kBatchFp32Polish ? r32.cycles : mode == sccs::kBatchFp32 ? r.cycles : 0;
        if (status == SCCS_OK && beta_out && beta_out[k] && h->d.J > 0)
            std::memcpy(beta_out[k], plan->res_beta_host + plan->beta_off[q], sizeof(double) * h->d.J);
        if (infos) {
            sccs_fit_info &fi = infos[k];
            const int32_t cyc = mode == sccs::kBatchFp32Polish ? fp32_cycles + r.cycles : r.cycles;
            fi.status = status != SCCS_OK ? status : r.status;
            fi.cycles = cyc;
            fi.steps = static_cast<int64_t>(cyc) * h->d.J;
            fi.nonzero_steps = r.nonzero_steps + (mode == sccs::kBatchFp32Polish ? r32.nonzero_steps : 0);
            fi.logpost = r.logpost;
            fi.conv_value = r.conv;
            fi.kernel_ms = kms;
            fi.total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
            fi.warnings = r.warnings | r32.warnings;
            fi.fp32_cycles = fp32_cycles;
        }
        if (status != SCCS_OK && first_err == SCCS_OK) first_err = status;
    }
    if (first_err != SCCS_OK) return fail(first_err, "at least one fit of the batch failed (see infos[k].status)");
    return SCCS_OK;
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

int sccs_heldout_loglik(sccs_handle *h, const double *beta, const int32_t *weights, double *loglik) {
    if (!h || !loglik) return fail(SCCS_E_INVAL, "null argument");
    int rc = set_device(h);
    if (rc) return rc;
    const int32_t J = h->d.J;
    int le = 0;
    if (beta) {
        for (int32_t j = 0; j < J; ++j)
            if (!std::isfinite(beta[j])) return fail(SCCS_E_INVAL, "beta has a non-finite entry");
        std::memcpy(h->beta_host, beta, sizeof(double) * static_cast<size_t>(J));
        cudaError_t e = cudaMemcpyAsync(h->beta_dev, h->beta_host, sizeof(double) * std::max<int32_t>(J, 1),
                                        cudaMemcpyHostToDevice, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync beta");
        // E and D rebuilt from beta in FP64, trust radii kept
        if ((rc = run_init_state(h, h->beta_dev, true))) return rc;
    } else if ((rc = refresh_fp64_state(h))) {
        return rc;
    }
    if (weights && (rc = prepare_weights(h, weights))) return rc;
    CountsScope counts(h, weights != nullptr);
    if (h->hist_cap < 1) {
        cudaError_t e = cudaMalloc(&h->hist_dev, sizeof(double));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc history");
        e = cudaMallocHost(&h->hist_host, sizeof(double));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocHost history");
        h->hist_cap = 1;
    }
    sccs::FitParams p = base_params(h);
    p.max_cycles = 0;
    le = sccs::launch_fit(h->d, p, h->out_dev, h->hist_dev, h->threads, h->stream);
    if (le != 0) return cuda_fail(static_cast<cudaError_t>(le), "fit kernel launch");
    if ((rc = sync_out(h))) return rc;
    const sccs::FitOut r = *h->out_host;
    if (r.status == -6 || r.abort_flag) {
        reset_after_abort(h);
        return fail(SCCS_E_TIMEOUT, "a device-side wait exceeded its bound; the handle was reset to beta = 0");
    }
    h->seq = r.seq_end;
    *loglik = r.loglik;
    return SCCS_OK;
}

int sccs_selftest_exp(int32_t device, const double *x, int64_t n, double *ours, double *ref) {
    if (n < 0 || (n > 0 && (!x || !ours || !ref))) return fail(SCCS_E_INVAL, "bad arguments");
    if (n == 0) return SCCS_OK;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    double *buf = nullptr;
    const size_t b = sizeof(double) * static_cast<size_t>(n);
    if (cudaMalloc(&buf, 3 * b) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(SCCS_E_NOMEM, "device buffers");
    }
    e = cudaMemcpy(buf, x, b, cudaMemcpyHostToDevice);
    int le = e == cudaSuccess ? sccs::launch_exp_selftest(buf, n, buf + n, buf + 2 * n, nullptr) : static_cast<int>(e);
    if (le == 0) e = cudaMemcpy(ours, buf + n, b, cudaMemcpyDeviceToHost);
    if (le == 0 && e == cudaSuccess) e = cudaMemcpy(ref, buf + 2 * n, b, cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (le != 0) return cuda_fail(static_cast<cudaError_t>(le), "exp self-test");
    if (e != cudaSuccess) return cuda_fail(e, "exp self-test copies");
    return SCCS_OK;
}

int sccs_selftest_div(int32_t device, const double *a, const double *b, int64_t n, double *ours, double *ref) {
    if (n < 0 || (n > 0 && (!a || !b || !ours || !ref))) return fail(SCCS_E_INVAL, "bad arguments");
    if (n == 0) return SCCS_OK;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    double *buf = nullptr;
    const size_t bytes = sizeof(double) * static_cast<size_t>(n);
    if (cudaMalloc(&buf, 4 * bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(SCCS_E_NOMEM, "device buffers");
    }
    e = cudaMemcpy(buf, a, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(buf + n, b, bytes, cudaMemcpyHostToDevice);
    int le = e == cudaSuccess ? sccs::launch_div_selftest(buf, buf + n, n, buf + 2 * n, buf + 3 * n, nullptr)
                              : static_cast<int>(e);
    if (le == 0) e = cudaMemcpy(ours, buf + 2 * n, bytes, cudaMemcpyDeviceToHost);
    if (le == 0 && e == cudaSuccess) e = cudaMemcpy(ref, buf + 3 * n, bytes, cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (le != 0) return cuda_fail(static_cast<cudaError_t>(le), "division self-test");
    if (e != cudaSuccess) return cuda_fail(e, "division self-test copies");
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
