// sccs_server.cpp -- a fit server: continuous batching of MAP-fit requests on one GPU.
//
// Datasets are created once with sccs_create and stay resident.  A request names a dataset
// and a prior (the cross-validation and bootstrap workflows of Section 2.5 issue many such
// fits per dataset).  Each admitted request runs in a "fit slot": device state of its own
// (L x exp(Xb), the denominators, beta and trust copies, all-reduce slots, stash) over the
// dataset's shared static layout, on a stream of its own.  A scheduler thread admits queued
// requests in arrival order whenever the slot memory fits the HBM budget and the request's
// CTA team fits next to the fits already running, so requests that arrive while others run
// start as soon as room frees up and their kernels overlap on the device.  A fit computes the
// same thing alone or in the mix: same layout, same team, fresh state.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sccs.h"
#include "sccs_internal.h"

namespace {

using Clock = std::chrono::steady_clock;
constexpr long long kWaitNs = 2000000000LL;
constexpr double kFp32PhaseRelTol = 1e-6;   // same switch point as sccs_fit

struct FitSlot {
    const sccs_handle *dataset = nullptr;
    sccs::DevLayout d{};
    const int32_t *base_nev = nullptr;  // the dataset's n_i and Y'X_j (unweighted requests)
    const double *base_ytx = nullptr;
    int32_t *w_dev = nullptr;           // N: a request's weights per kept subject
    int32_t *nev_w = nullptr;           // N: w_i n_i
    double *ytx_w = nullptr;            // J: weighted Y'X_j
    int32_t *nev_ho = nullptr;          // N: held-out counts (evaluated inside the fit kernel)
    double *ytx_ho = nullptr;           // J
    int32_t *w_host = nullptr;          // 2N pinned: training weights, then held-out weights
    sccs::FitOut *out_ho_dev = nullptr; // held-out evaluation
    sccs::FitOut *out_ho_host = nullptr;
    int threads = 512;
    size_t bytes = 0;
    void *block = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    sccs::FitOut *out_dev = nullptr;
    sccs::FitOut *out_host = nullptr;   // pinned
    double *beta_host = nullptr;        // pinned, J
    double *beta_dev = nullptr;
    double *hist_dev = nullptr;
    int hist_cap = 0;
    unsigned long long seq = 0;
};

struct Request {
    uint64_t ticket = 0;
    sccs_handle *dataset = nullptr;     // the handle the fit runs on (chosen at admission)
    sccs_handle *small = nullptr;       // the smaller-team handle of the request (or its only one)
    sccs_handle *large = nullptr;       // the larger-team handle, or null
    int S_small = 0, S_large = 0;
    int prior = SCCS_PRIOR_NONE;
    double variance = 1.0;
    int tol_mode = SCCS_TOL_REL_LOGPOST;
    double tol = 1e-12;
    int max_cycles = 1000;
    int precision = SCCS_PREC_FP64;
    std::vector<double> beta0;
    std::vector<int32_t> w_train, w_ho;   // per kept subject (empty: none)
    double heldout_loglik = std::nan("");
    int J = 0;
    int S = 0;
    Clock::time_point t_submit, t_start, t_done;
    FitSlot *slot = nullptr;
    int phase = 0;                      // 0 queued, 1 FP32 phase, 2 FP64 phase, 3 done
    int fp32_cycles = 0;
    int status = SCCS_OK;
    int cycles = 0;
    double logpost = 0.0;
    std::vector<double> beta;
    bool cancelled = false;
};

size_t slot_bytes(const sccs::DevLayout &d, int max_cycles) {
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t K = static_cast<size_t>(d.K), N = static_cast<size_t>(d.N), S = d.S,
                 J = static_cast<size_t>(std::max(d.J, 1));
    const size_t N1 = std::max<size_t>(N, 1);
    return al(8 * K) + al(8 * N) + al(4 * K) + al(8 * N) + 2 * al(8 * S * J) +
           al(16 * S * static_cast<size_t>(d.stash_stride)) + al(32 * S) + 2 * al(sizeof(sccs::FitOut)) +
           al(8 * J) + al(8 * static_cast<size_t>(max_cycles + 1)) + 3 * al(4 * N1) + 2 * al(8 * J) + al(256) + al(8 * K) +
           al(8 * S * static_cast<size_t>(d.estash_stride));
}

}  // namespace

struct sccs_server {
    int device = 0;
    int max_inflight = 64;
    int queue_capacity = 4096;
    long long budget = 0;
    int capacity_ctas = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request *> pending;
    std::vector<Request *> running;
    std::unordered_map<uint64_t, Request *> tickets;   // every live ticket
    std::vector<FitSlot *> idle;                       // slots with no request, any dataset
    long long allocated = 0;
    int ctas_in_use = 0;
    uint64_t next_ticket = 1;
    uint64_t completed = 0;
    bool stop = false;
    std::thread worker;
    std::string fatal;
};

namespace {

void free_slot(FitSlot *s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->block) cudaFree(s->block);
    if (s->hist_dev) cudaFree(s->hist_dev);
    if (s->out_host) cudaFreeHost(s->out_host);
    if (s->beta_host) cudaFreeHost(s->beta_host);
    if (s->w_host) cudaFreeHost(s->w_host);
    if (s->out_ho_host) cudaFreeHost(s->out_ho_host);
    if (s->done) cudaEventDestroy(s->done);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

// Device state for one fit of `dataset` (static arrays shared with the dataset handle).
FitSlot *make_slot(const sccs_handle *dataset, int max_cycles) {
    sccs::HandleView v{};
    if (!sccs_handle_view(dataset, &v)) return nullptr;
    FitSlot *s = new FitSlot();
    s->dataset = dataset;
    s->threads = v.threads;
    s->d = v.d;
    s->base_nev = v.d.nev;
    s->base_ytx = v.d.ytx;
    sccs::DevLayout &d = s->d;
    const size_t bytes = slot_bytes(d, 0);
    s->bytes = bytes;
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
        (void)cudaGetLastError();
        s->stream = nullptr;
        free_slot(s);
        return nullptr;
    }
    if (cudaMalloc(&s->block, bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        s->block = nullptr;
        free_slot(s);
        return nullptr;
    }
    // zeroed on the slot's own stream, ahead of its first kernel
    cudaMemsetAsync(s->block, 0, bytes, s->stream);
    char *p = static_cast<char *>(s->block);
    auto take = [&](size_t b) {
        char *q = p;
        p += (b + 255) / 256 * 256;
        return q;
    };
    const size_t K = static_cast<size_t>(d.K), N = static_cast<size_t>(d.N), S = d.S,
                 J = static_cast<size_t>(std::max(d.J, 1));
    d.E = reinterpret_cast<double *>(take(8 * K));
    d.D = reinterpret_cast<double *>(take(8 * N));
    d.E32 = reinterpret_cast<float *>(take(4 * K));
    d.D32 = reinterpret_cast<float2 *>(take(8 * N));
    d.beta_priv = reinterpret_cast<double *>(take(8 * S * J));
    d.trust_priv = reinterpret_cast<double *>(take(8 * S * J));
    d.stash = reinterpret_cast<double *>(take(16 * S * static_cast<size_t>(d.stash_stride)));
    d.slots = reinterpret_cast<unsigned long long *>(take(32 * S));
    s->out_dev = reinterpret_cast<sccs::FitOut *>(take(sizeof(sccs::FitOut)));
    s->out_ho_dev = reinterpret_cast<sccs::FitOut *>(take(sizeof(sccs::FitOut)));
    s->beta_dev = reinterpret_cast<double *>(take(8 * J));
    const size_t N1 = std::max<size_t>(N, 1);
    s->w_dev = reinterpret_cast<int32_t *>(take(4 * N1));
    s->nev_w = reinterpret_cast<int32_t *>(take(4 * N1));
    s->ytx_w = reinterpret_cast<double *>(take(8 * J));
    s->nev_ho = reinterpret_cast<int32_t *>(take(4 * N1));
    auto *nsync = reinterpret_cast<unsigned long long *>(take(256));
    d.E_prev = reinterpret_cast<double *>(take(8 * std::max<size_t>(K, 1)));   // Genkin's X-beta test
    if (d.narrow) d.nar_sync = nsync;   // the slot's own narrow-run counters
    if (d.C > 0) d.clu_sync = nsync + 8;   // and cluster-run counters ([8] and [24] of the same 256 bytes)
    s->ytx_ho = reinterpret_cast<double *>(take(8 * J));
    d.estash = reinterpret_cast<double *>(take(8 * S * static_cast<size_t>(d.estash_stride)));
    d.abort_flag = &s->out_dev->abort_flag;
    if (cudaEventCreateWithFlags(&s->done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(&s->out_host, sizeof(sccs::FitOut)) != cudaSuccess ||
        cudaMallocHost(&s->out_ho_host, sizeof(sccs::FitOut)) != cudaSuccess ||
        cudaMallocHost(&s->w_host, 8 * N1) != cudaSuccess ||
        cudaMallocHost(&s->beta_host, 8 * J) != cudaSuccess) {
        (void)cudaGetLastError();
        free_slot(s);
        return nullptr;
    }
    (void)max_cycles;
    return s;
}

bool ensure_hist(FitSlot *s, int max_cycles) {
    if (s->hist_cap >= max_cycles + 1) return true;
    if (s->hist_dev) cudaFree(s->hist_dev);
    s->hist_dev = nullptr;
    s->hist_cap = 0;
    if (cudaMalloc(&s->hist_dev, sizeof(double) * (max_cycles + 1)) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    s->hist_cap = max_cycles + 1;
    return true;
}

sccs::FitParams params_for(const Request &r, const FitSlot &s, bool fp32_phase) {
    sccs::FitParams p{};
    p.prior = r.prior;
    p.variance = r.prior == SCCS_PRIOR_NONE ? 1.0 : r.variance;
    p.inv_var = 1.0 / p.variance;
    p.lambda = r.prior == SCCS_PRIOR_LAPLACE ? std::sqrt(2.0 / r.variance) : 0.0;
    p.tol_mode = r.tol_mode;
    p.tol = r.tol;
    p.max_cycles = r.max_cycles;
    p.record_history = 1;
    p.seq0 = s.seq;
    p.timeout_ns = kWaitNs;
    if (fp32_phase && r.precision == SCCS_PREC_FP32_POLISH) {
        p.tol_mode = SCCS_TOL_REL_LOGPOST;
        p.tol = kFp32PhaseRelTol;
    }
    return p;
}

// Enqueue one phase of a request on its slot's stream; completion is signalled by slot->done.
int enqueue_phase(Request &r, bool first) {
    FitSlot &s = *r.slot;
    const bool fp32 = r.phase == 1;
    const bool final_phase = !(r.phase == 1 && r.precision == SCCS_PREC_FP32_POLISH);
    const size_t N1 = static_cast<size_t>(std::max<int64_t>(s.d.N, 1));
    // weighted counts are always formed from the dataset's own n_i and Y'X_j pairs
    sccs::DevLayout base = s.d;
    base.nev = s.base_nev;
    base.ytx = s.base_ytx;
    int e = 0;
    if (first) {
        // the request's counts: weighted (Section 2.5) or the dataset's own
        if (!r.w_train.empty()) {
            std::memcpy(s.w_host, r.w_train.data(), sizeof(int32_t) * r.w_train.size());
            cudaMemcpyAsync(s.w_dev, s.w_host, sizeof(int32_t) * N1, cudaMemcpyHostToDevice, s.stream);
            e = sccs::launch_weighted_counts(base, s.w_dev, s.nev_w, s.ytx_w, s.stream);
            if (e) return e;
            s.d.nev = s.nev_w;
            s.d.ytx = s.ytx_w;
        } else {
            s.d.nev = s.base_nev;
            s.d.ytx = s.base_ytx;
        }
        if (!r.w_ho.empty() && r.precision != SCCS_PREC_FP32) {
            // held-out counts now; the final FP64 phase evaluates them before it returns
            int32_t *wh = s.w_host + N1;
            std::memcpy(wh, r.w_ho.data(), sizeof(int32_t) * r.w_ho.size());
            cudaMemcpyAsync(s.w_dev, wh, sizeof(int32_t) * N1, cudaMemcpyHostToDevice, s.stream);
            e = sccs::launch_weighted_counts(base, s.w_dev, s.nev_ho, s.ytx_ho, s.stream);
            if (e) return e;
        }
        if (!r.beta0.empty()) {
            std::memcpy(s.beta_host, r.beta0.data(), sizeof(double) * r.J);
            cudaMemcpyAsync(s.beta_dev, s.beta_host, sizeof(double) * r.J, cudaMemcpyHostToDevice, s.stream);
            e = sccs::launch_init_state(s.d, s.beta_dev, s.threads, s.stream);
        } else {
            e = sccs::launch_init_state(s.d, nullptr, s.threads, s.stream);
        }
        if (!e && fp32) e = sccs::launch_e_to_f32(s.d, s.threads, s.stream);
    } else {
        // FP64 polish from the FP32 point: E and D rebuilt in FP64, trust radii kept
        cudaMemcpyAsync(s.beta_dev, s.d.beta_priv, sizeof(double) * std::max(r.J, 1), cudaMemcpyDeviceToDevice,
                        s.stream);
        e = sccs::launch_init_state(s.d, s.beta_dev, s.threads, s.stream, true);
    }
    if (e) return e;
    sccs::FitParams p = params_for(r, s, fp32);
    if (final_phase && !fp32 && !r.w_ho.empty()) {
        p.ho_nev = s.nev_ho;
        p.ho_ytx = s.ytx_ho;
    }
    e = sccs::launch_fit(s.d, p, s.out_dev, s.hist_dev, s.threads, s.stream, fp32);
    if (e) return e;
    cudaMemcpyAsync(s.out_host, s.out_dev, sizeof(sccs::FitOut), cudaMemcpyDeviceToHost, s.stream);
    if (r.J > 0) cudaMemcpyAsync(s.beta_host, s.d.beta_priv, sizeof(double) * r.J, cudaMemcpyDeviceToHost, s.stream);
    if (final_phase && !r.w_ho.empty() && r.precision == SCCS_PREC_FP32) {
        // FP32-only fit: the held-out predictive log-likelihood by a separate FP64 evaluation
        // at the fitted beta (as sccs_heldout_loglik)
        int32_t *wh = s.w_host + N1;
        std::memcpy(wh, r.w_ho.data(), sizeof(int32_t) * r.w_ho.size());
        cudaMemcpyAsync(s.w_dev, wh, sizeof(int32_t) * N1, cudaMemcpyHostToDevice, s.stream);
        e = sccs::launch_weighted_counts(base, s.w_dev, s.nev_w, s.ytx_w, s.stream);
        if (e) return e;
        sccs::DevLayout dh = s.d;
        dh.nev = s.nev_w;
        dh.ytx = s.ytx_w;
        // the FP32-only fit kept E in FP32: rebuild the FP64 state from its beta first
        cudaMemcpyAsync(s.beta_dev, s.d.beta_priv, sizeof(double) * std::max(r.J, 1), cudaMemcpyDeviceToDevice,
                        s.stream);
        e = sccs::launch_init_state(dh, s.beta_dev, s.threads, s.stream, true);
        if (e) return e;
        sccs::FitParams ph = params_for(r, s, false);
        ph.max_cycles = 0;
        ph.seq_src = &s.out_dev->seq_end;   // continues where the fit's all-reduces ended
        e = sccs::launch_fit(dh, ph, s.out_ho_dev, s.hist_dev, s.threads, s.stream, false);
        if (e) return e;
        cudaMemcpyAsync(s.out_ho_host, s.out_ho_dev, sizeof(sccs::FitOut), cudaMemcpyDeviceToHost, s.stream);
    }
    return static_cast<int>(cudaEventRecord(s.done, s.stream));
}

void reset_slot_after_abort(FitSlot &s) {
    cudaStreamSynchronize(s.stream);
    cudaMemsetAsync(s.d.slots, 0, 32 * static_cast<size_t>(s.d.S), s.stream);
    cudaMemsetAsync(s.out_dev, 0, sizeof(sccs::FitOut), s.stream);
    cudaStreamSynchronize(s.stream);
    s.seq = 0;
}

// Take an idle slot for the request's dataset, or make one if the budget allows (evicting
// idle slots of other datasets when needed).  Called with the server lock held.
FitSlot *acquire_slot(sccs_server *sv, Request &r) {
    for (size_t i = 0; i < sv->idle.size(); ++i) {
        if (sv->idle[i]->dataset == r.dataset) {
            FitSlot *s = sv->idle[i];
            sv->idle.erase(sv->idle.begin() + static_cast<long>(i));
            return s;
        }
    }
    sccs::HandleView v{};
    sccs_handle_view(r.dataset, &v);
    const long long need = static_cast<long long>(slot_bytes(v.d, 0));
    while (sv->budget > 0 && sv->allocated + need > sv->budget && !sv->idle.empty()) {
        FitSlot *old = sv->idle.front();
        sv->idle.erase(sv->idle.begin());
        sv->allocated -= static_cast<long long>(old->bytes);
        free_slot(old);
    }
    if (sv->budget > 0 && sv->allocated + need > sv->budget) return nullptr;
    FitSlot *s = make_slot(r.dataset, r.max_cycles);
    if (s) sv->allocated += static_cast<long long>(s->bytes);
    return s;
}

void finish(sccs_server *sv, Request *r, int status) {
    r->status = status;
    r->t_done = Clock::now();
    r->phase = 3;
    FitSlot *s = r->slot;
    if (s) {
        sv->ctas_in_use -= r->S;
        sv->idle.push_back(s);
        r->slot = nullptr;
    }
    sv->completed++;
}

void worker_main(sccs_server *sv) {
    cudaSetDevice(sv->device);
    std::vector<Request *> to_launch;
    for (;;) {
        to_launch.clear();
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            if (sv->pending.empty() && sv->running.empty()) {
                if (sv->stop) break;
                sv->cv.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
            // admission in arrival order
            while (!sv->pending.empty() && static_cast<int>(sv->running.size()) < sv->max_inflight) {
                Request *r = sv->pending.front();
                if (r->cancelled) {
                    sv->pending.pop_front();
                    finish(sv, r, SCCS_E_INVAL);
                    continue;
                }
                // an idle device and nothing else waiting: the larger team, for latency
                const bool go_large = r->large && sv->running.empty() && sv->pending.size() == 1;
                r->dataset = go_large ? r->large : r->small;
                r->S = go_large ? r->S_large : r->S_small;
                if (sv->ctas_in_use + r->S > sv->capacity_ctas && !sv->running.empty()) break;
                FitSlot *s = acquire_slot(sv, *r);
                if (!s && go_large) {       // the larger team's state does not fit the budget
                    r->dataset = r->small;
                    r->S = r->S_small;
                    s = acquire_slot(sv, *r);
                }
                if (!s) {
                    if (sv->running.empty()) {   // it will never fit
                        sv->pending.pop_front();
                        finish(sv, r, SCCS_E_NOMEM);
                        continue;
                    }
                    break;
                }
                if (!ensure_hist(s, r->max_cycles)) {
                    sv->idle.push_back(s);
                    sv->pending.pop_front();
                    finish(sv, r, SCCS_E_NOMEM);
                    continue;
                }
                sv->pending.pop_front();
                r->slot = s;
                r->t_start = Clock::now();
                r->phase = r->precision == SCCS_PREC_FP64 ? 2 : 1;
                sv->ctas_in_use += r->S;
                sv->running.push_back(r);
                to_launch.push_back(r);
            }
        }
        for (Request *r : to_launch) {
            if (enqueue_phase(*r, true)) {
                (void)cudaGetLastError();
                std::lock_guard<std::mutex> lk(sv->mu);
                reset_slot_after_abort(*r->slot);
                sv->running.erase(std::find(sv->running.begin(), sv->running.end(), r));
                finish(sv, r, SCCS_E_CUDA);
            }
        }
        // progress of running fits
        bool progressed = !to_launch.empty();
        std::vector<Request *> snapshot;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            snapshot = sv->running;
        }
        for (Request *r : snapshot) {
            FitSlot &s = *r->slot;
            const cudaError_t q = cudaEventQuery(s.done);
            if (q == cudaErrorNotReady) continue;
            progressed = true;
            const sccs::FitOut out = *s.out_host;
            const bool final_phase = !(r->phase == 1 && r->precision == SCCS_PREC_FP32_POLISH);
            const bool heldout = final_phase && !r->w_ho.empty();
            const bool heldout_apart = heldout && r->precision == SCCS_PREC_FP32;   // a second launch
            const sccs::FitOut out_ho = heldout_apart ? *s.out_ho_host : sccs::FitOut{};
            int status = SCCS_OK;
            if (q != cudaSuccess) {
                (void)cudaGetLastError();
                status = SCCS_E_CUDA;
            } else if (out.status == -6 || out.abort_flag ||
                       (heldout_apart && (out_ho.status == -6 || out_ho.abort_flag))) {
                status = SCCS_E_TIMEOUT;
            } else if (out.status == -7 || (heldout_apart && out_ho.status == -7)) {
                status = SCCS_E_NUMERIC;
            }
            if (status == SCCS_OK) s.seq = heldout_apart ? out_ho.seq_end : out.seq_end;
            else reset_slot_after_abort(s);
            if (status == SCCS_OK && r->phase == 1 && r->precision == SCCS_PREC_FP32_POLISH) {
                {
                    std::lock_guard<std::mutex> lk(sv->mu);
                    r->fp32_cycles = out.cycles;
                    r->phase = 2;
                }
                if (enqueue_phase(*r, false) == 0) continue;
                (void)cudaGetLastError();
                status = SCCS_E_CUDA;
            }
            std::lock_guard<std::mutex> lk(sv->mu);
            if (status == SCCS_OK) {
                r->cycles = out.cycles + (r->precision == SCCS_PREC_FP32_POLISH ? r->fp32_cycles : 0);
                if (r->precision == SCCS_PREC_FP32) r->fp32_cycles = out.cycles;
                r->logpost = out.logpost;
                r->heldout_loglik = !heldout ? std::nan("") : heldout_apart ? out_ho.loglik : out.heldout_loglik;
                r->beta.assign(s.beta_host, s.beta_host + r->J);
                status = out.status == 0 ? SCCS_OK : SCCS_NOT_CONVERGED;
            }
            sv->running.erase(std::find(sv->running.begin(), sv->running.end(), r));
            finish(sv, r, status);
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

}  // namespace

extern "C" {

int sccs_server_create(sccs_server **out, const sccs_server_opts *opts) {
    if (!out) return sccs_set_error(SCCS_E_INVAL, "out is null");
    *out = nullptr;
    sccs_server_opts o{};
    o.struct_size = sizeof(sccs_server_opts);
    o.max_inflight = 64;
    o.queue_capacity = 4096;
    if (opts) {
        if (opts->struct_size != static_cast<int32_t>(sizeof(sccs_server_opts)))
            return sccs_set_error(SCCS_E_INVAL, "sccs_server_opts.struct_size mismatch");
        o = *opts;
    }
    if (o.max_inflight < 1 || o.queue_capacity < 1 || o.hbm_budget_bytes < 0)
        return sccs_set_error(SCCS_E_INVAL, "max_inflight and queue_capacity must be >= 1, the budget >= 0");
    cudaError_t e = cudaSetDevice(o.device);
    if (e != cudaSuccess) return sccs_set_error(SCCS_E_CUDA, cudaGetErrorString(e));
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, o.device);
    int rc = sccs::fit_kernel_max_blocks_per_sm(512, &per_sm);
    if (rc) return sccs_set_error(SCCS_E_CUDA, "occupancy query failed");
    sccs_server *sv = new sccs_server();
    sv->device = o.device;
    sv->max_inflight = o.max_inflight;
    sv->queue_capacity = o.queue_capacity;
    sv->budget = o.hbm_budget_bytes;
    sv->capacity_ctas = sms * std::max(per_sm, 1);
    sv->worker = std::thread(worker_main, sv);
    *out = sv;
    return SCCS_OK;
}

int sccs_submit(sccs_server *sv, const sccs_request *req, uint64_t *ticket) {
    if (!sv || !req || !ticket) return sccs_set_error(SCCS_E_INVAL, "null argument");
    if (req->struct_size != static_cast<int32_t>(sizeof(sccs_request)))
        return sccs_set_error(SCCS_E_INVAL, "sccs_request.struct_size mismatch");
    sccs::HandleView v{};
    if (!sccs_handle_view(req->dataset, &v)) return sccs_set_error(SCCS_E_INVAL, "request without a dataset");
    if (v.device != sv->device) return sccs_set_error(SCCS_E_INVAL, "dataset on another device");
    if (req->prior_type != SCCS_PRIOR_NONE && req->prior_type != SCCS_PRIOR_NORMAL &&
        req->prior_type != SCCS_PRIOR_LAPLACE)
        return sccs_set_error(SCCS_E_INVAL, "unknown prior type");
    if (req->prior_type != SCCS_PRIOR_NONE && !(req->variance > 0.0 && std::isfinite(req->variance)))
        return sccs_set_error(SCCS_E_INVAL, "prior variance must be positive and finite");
    if (req->tol_mode != SCCS_TOL_ABS_LOGPOST && req->tol_mode != SCCS_TOL_REL_LOGPOST &&
        req->tol_mode != SCCS_TOL_GENKIN_XBETA)
        return sccs_set_error(SCCS_E_INVAL, "unknown tol_mode");
    if (req->tol_mode == SCCS_TOL_GENKIN_XBETA && req->precision == SCCS_PREC_FP32)
        return sccs_set_error(SCCS_E_UNSUPPORTED, "the Genkin X-beta test needs the FP64 state");
    if (req->max_cycles < 0) return sccs_set_error(SCCS_E_INVAL, "max_cycles must be >= 0");
    if (req->precision != SCCS_PREC_FP64 && req->precision != SCCS_PREC_FP32_POLISH &&
        req->precision != SCCS_PREC_FP32)
        return sccs_set_error(SCCS_E_INVAL, "unknown precision");
    if (v.d.S > sv->capacity_ctas) return sccs_set_error(SCCS_E_INVAL, "dataset has more shards than the device holds");
    sccs::HandleView va{};
    if (req->dataset_alt) {
        if (!sccs_handle_view(req->dataset_alt, &va)) return sccs_set_error(SCCS_E_INVAL, "bad dataset_alt");
        if (va.device != v.device || va.d.J != v.d.J || va.d.K != v.d.K || va.d.N != v.d.N ||
            va.subjects_in != v.subjects_in)
            return sccs_set_error(SCCS_E_INVAL, "dataset_alt does not hold the same data as dataset");
        if (va.d.S > sv->capacity_ctas) return sccs_set_error(SCCS_E_INVAL, "dataset_alt has more shards than the device holds");
    }
    Request *r = new Request();
    r->dataset = req->dataset;
    r->small = req->dataset;
    r->S_small = v.d.S;
    if (req->dataset_alt && req->dataset_alt != req->dataset) {
        if (va.d.S >= v.d.S) {
            r->large = req->dataset_alt;
            r->S_large = va.d.S;
        } else {
            r->large = req->dataset;
            r->S_large = v.d.S;
            r->small = req->dataset_alt;
            r->S_small = va.d.S;
        }
    }
    r->prior = req->prior_type;
    r->variance = req->variance;
    r->tol_mode = req->tol_mode;
    r->tol = req->tol;
    r->max_cycles = req->max_cycles;
    r->precision = req->precision;
    r->J = v.d.J;
    r->S = v.d.S;
    if (req->beta0) {
        for (int j = 0; j < r->J; ++j)
            if (!std::isfinite(req->beta0[j])) {
                delete r;
                return sccs_set_error(SCCS_E_INVAL, "beta0 has a non-finite entry");
            }
        r->beta0.assign(req->beta0, req->beta0 + r->J);
    }
    // Section 2.5 weights, mapped to kept subjects now (the caller's arrays need not outlive this call)
    for (int which = 0; which < 2; ++which) {
        const int32_t *w_in = which == 0 ? req->subject_weights : req->heldout_weights;
        if (!w_in) continue;
        std::vector<int32_t> &w = which == 0 ? r->w_train : r->w_ho;
        w.assign(static_cast<size_t>(std::max<int64_t>(v.d.N, 1)), 0);
        const int rc = sccs::map_subject_weights(v, w_in, w.data());
        if (rc != SCCS_OK) {
            delete r;
            return rc;
        }
    }
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stop) {
            delete r;
            return sccs_set_error(SCCS_E_INVAL, "server is shutting down");
        }
        if (static_cast<int>(sv->pending.size()) >= sv->queue_capacity) {
            delete r;
            return sccs_set_error(SCCS_E_BUSY, "request queue is full");
        }
        r->ticket = sv->next_ticket++;
        sv->tickets[r->ticket] = r;
        sv->pending.push_back(r);
        *ticket = r->ticket;
    }
    sv->cv.notify_one();
    return SCCS_OK;
}

int sccs_poll(sccs_server *sv, uint64_t ticket, sccs_result *res) {
    if (!sv || !res) return sccs_set_error(SCCS_E_INVAL, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->tickets.find(ticket);
    if (it == sv->tickets.end()) return sccs_set_error(SCCS_E_INVAL, "unknown or already collected ticket");
    Request *r = it->second;
    if (r->phase != 3) return SCCS_PENDING;
    res->status = r->status;
    res->team = r->S;
    res->cycles = r->cycles;
    res->fp32_cycles = r->fp32_cycles;
    res->logpost = r->logpost;
    res->heldout_loglik = r->status == SCCS_OK || r->status == SCCS_NOT_CONVERGED ? r->heldout_loglik : std::nan("");
    res->queue_ms = std::chrono::duration<double, std::milli>(r->t_start - r->t_submit).count();
    res->latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    if (r->phase == 3 && r->t_start < r->t_submit) res->queue_ms = 0.0;
    if (res->beta && !r->beta.empty()) std::memcpy(res->beta, r->beta.data(), sizeof(double) * r->beta.size());
    sv->tickets.erase(it);
    delete r;
    return SCCS_OK;
}

int sccs_server_get_stats(sccs_server *sv, sccs_server_stats *st) {
    if (!sv || !st) return sccs_set_error(SCCS_E_INVAL, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    st->pending = static_cast<int64_t>(sv->pending.size());
    st->running = static_cast<int64_t>(sv->running.size());
    st->completed = static_cast<int64_t>(sv->completed);
    st->slot_bytes = sv->allocated;
    st->ctas_in_use = sv->ctas_in_use;
    st->capacity_ctas = sv->capacity_ctas;
    return SCCS_OK;
}

int sccs_server_destroy(sccs_server *sv) {
    if (!sv) return SCCS_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        for (Request *r : sv->pending) r->cancelled = true;
    }
    sv->cv.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    cudaSetDevice(sv->device);
    for (FitSlot *s : sv->idle) free_slot(s);
    for (auto &kv : sv->tickets) delete kv.second;
    delete sv;
    return SCCS_OK;
}

}  // extern "C"
