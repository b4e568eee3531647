// sccs_internal.h -- device layout shared by the host set-up code and the CUDA kernels.
//
// Layout ("subject shards"): the kept rows are cut into S contiguous shards at subject
// boundaries; shard s is owned by CTA s of every kernel, which alone reads and writes
// L x exp(Xb) (E) on the shard's rows and M[L x exp(Xb)] (D) on its subjects.  The
// only data CTAs exchange is the pair of partial sums per coordinate (Eqs. 7-9 are sums
// over subjects), so a coordinate step needs one grid-wide all-reduce and no other barrier.
//
// Each column X_j is split into per-shard slices.  A slice's nonzeros are grouped by subject
// into "segments" (the paper's COO rows of M X_j, Section 2.3), ordered by length, longest
// first, and packed 32 to a group.  A group stores its rows diagonal by diagonal (jagged
// diagonal order): diagonal t holds the t-th row of every segment longer than t, so the
// lanes active at step t are exactly the first c_t lanes and every step is one coalesced
// load.  A lane then owns one whole segment and sums its numerator with no cross-lane
// traffic.
#pragma once

#include <cstddef>
#include <cstdint>

#include <vector_types.h>

namespace sccs {

constexpr int kMaxShards = 4096;
constexpr int kWarp = 32;

// Slices up to these sizes are staged in shared memory by bulk copies one column ahead.
constexpr int kSegCap = 2048;              // segments per staged slice
constexpr int kRowCap = 4096;              // nonzeros per staged slice
constexpr int kGrpCap = kSegCap / 32;      // groups per staged slice
constexpr int kNarrowGroupMax = 8;         // narrow columns whose steps are taken side by side
constexpr int kNarrowAfterWide = kNarrowGroupMax + 1;  // segment mark: waits on the wide column before the run
// Global arrays read by bulk copies are padded by this many bytes past their end, so a copy
// rounded out to 16-byte boundaries stays inside the allocation.
constexpr int kCopyPad = 32;

struct DevLayout {
    int32_t S;                 // shards == CTAs
    int32_t J;                 // columns
    int64_t K;                 // kept rows
    int64_t N;                 // kept subjects
    // static structure
    const int32_t *rows;       // JDS row index per nonzero (global kept-row id)
    const int2 *segs;          // per segment: {subject id, length}
    const int64_t *grp_base;   // per group: index into rows[] of its first diagonal
    const int64_t *slice_row;  // S*(J+1): first rows[] index of slice (s, j)
    const int64_t *slice_seg;  // S*(J+1): first segment of slice (s, j)
    const int64_t *slice_grp;  // S*(J+1): first group of slice (s, j)
    const int64_t *shard_row;  // S+1
    const int64_t *shard_pat;  // S+1
    const int64_t *pat_ptr;    // N+1: rows of subject i
    const int32_t *nev;        // N: n_i (or w_i n_i in a weighted fit)
    const double *L;           // K: offsets l_k
    const double *ytx;         // J: Y'X_j (or its weighted form)
    // narrow columns: whole column on the team's CTA 0 with block-level sums (null: none)
    const uint8_t *narrow;     // J: 1 for a narrow column
    const int32_t *next_wide;  // J: the next wide column after j, cyclically
    int32_t first_wide;        // first wide column (-1: none)
    int32_t pad_nw;
    const int64_t *nar_ptr;    // J+1: a narrow column's segments in nar_seg
    const int4 *nar_seg;       //   {subject, rows, first row in nar_row, 0}, subjects ascending
    const int32_t *nar_row;    //   rows of each segment, ascending
    const int32_t *nar_group;  // J: columns in the group starting at j (0 inside a group)
    unsigned long long *nar_sync;  // per fit state: [0] CTAs arrived at a narrow run, [16] runs done
    const int64_t *row_ptr;    // K+1: row -> columns index (built on the device at create)
    const int32_t *row_col;    //   the columns of each row, ascending
    const int64_t *ycol_ptr;   // J+1: per column, its (subject, sum of y) pairs with events
    const int32_t *ysub;       //   kept subject of each pair
    const int32_t *ycnt;       //   sum of y over the column's rows of that subject
    // cluster columns (FP64 fits launched with thread-block clusters of C CTAs): a column with
    // ccls[j] = 1 runs on the C CTAs of the first cluster, CTA c over its own subject shard c of a
    // second partition (slices cslice_*), with the partial sums reduced through distributed
    // shared memory instead of the grid all-reduce.  C = 0: no cluster columns.
    int32_t C;
    int32_t first_grid;        // first column run by the whole team (-1: none)
    const uint8_t *ccls;       // J
    const int32_t *next_grid;  // J: the next column run by the whole team after j, cyclically
    const int32_t *cgroup;     // J: columns in the cluster group starting at j (0 inside a group):
                               //    consecutive cluster columns with pairwise disjoint subjects
    const int32_t *crows;      // as rows / segs / grp_base, over the C shards
    const int2 *csegs;
    const int64_t *cgrp_base;
    const int64_t *cslice_row; // C*(J+1)
    const int64_t *cslice_seg;
    const int64_t *cslice_grp;
    unsigned long long *clu_sync;  // per fit state: [0] CTAs arrived at a cluster run, [16] runs done
    // state
    double *E;                 // K: L x exp(Xb)
    double *E_prev;            // K: E at the start of the cycle (Genkin's X-beta rule), or null
    double *D;                 // N: M[L x exp(Xb)]
    float *E32;                // K: L x exp(Xb) in the FP32 mode
    float2 *D32;               // N: M[L x exp(Xb)] as an FP32 (hi, lo) pair in the FP32 mode
    double *beta_priv;         // S*J: each CTA's private copy of beta (all copies agree)
    double *trust_priv;        // S*J: each CTA's private trust radii
    double *stash;             // S*stash_stride*2: (num, D) per segment of slices too big to stage
    int64_t stash_stride;      // segments per shard
    double *estash;            // S*estash_stride: E per row of slices too big to stage, phase A -> C
    int64_t estash_stride;     // rows per shard (the largest slice)
    // grid all-reduce slots: 2 buffers x S slots x {a, b}; sign bit carries the phase
    unsigned long long *slots;
    int *abort_flag;           // set by a CTA that gives up; every wait checks it (lives in FitOut)
};

struct FitParams {
    int32_t prior;             // SCCS_PRIOR_*
    int32_t tol_mode;
    double variance;
    double inv_var;            // 1 / variance
    double lambda;             // Laplace sqrt(2/variance)
    double tol;
    int32_t max_cycles;
    int32_t record_history;
    unsigned long long seq0;   // all-reduce sequence number at launch
    long long timeout_ns;      // bound on each device-side wait (from the start of that wait)
    const unsigned long long *seq_src;  // device; if set, seq0 is read from here at launch (the
                                        // seq_end of the launch before it on the same stream)
    const int32_t *ho_nev;     // device [N] or null: held-out counts w_i n_i (FP64 fits only); the
    const double *ho_ytx;      // [J] fit then ends with Eq. 2 under them in out->heldout_loglik
    int32_t cluster;           // 1: launched in clusters of DevLayout::C CTAs (cluster columns on)
    int32_t regather_e;        // 1: phase C of slices too big to stage gathers E again (from L2)
                               //    instead of reading the E stash phase A wrote
};

struct FitOut {
    double logpost;
    double conv;
    double loglik;
    int32_t cycles;
    int32_t status;            // 0 ok, 1 not converged, negative error
    int64_t nonzero_steps;
    int32_t warnings;
    int32_t err_where;         // diagnostic: which wait timed out
    unsigned long long seq_end;
    double g, h;               // grad_hess output
    int32_t abort_flag;        // nonzero if any CTA gave up a wait
    int32_t pad;
    double heldout_loglik;     // with FitParams::ho_nev: the held-out predictive log-likelihood
};

// One fit of a batched launch: its layout and state, parameters and outputs.  p32 drives
// the FP32 phase (FP32 and FP32-then-polish), p the FP64 fit or polish.  out receives the
// fit's final result; out32 the FP32 phase's when a polish follows it.
struct BatchEntry {
    DevLayout d;
    FitParams p;
    FitParams p32;
    FitOut *out;
    FitOut *out32;
    double *hist;
    int32_t warm;              // start from the handle's current beta instead of 0
    int32_t team;              // d.S: CTAs that run this fit together
};

// Precision of a batched launch.
enum BatchMode : int { kBatchFp64 = 0, kBatchFp32Polish = 1, kBatchFp32 = 2 };

// Dynamic shared memory the fit kernel needs.
size_t fit_kernel_smem_bytes();

// Launchers (return cudaError_t as int).  `stream` is a cudaStream_t.
// E = L x exp(X beta0) (beta0 = nullptr: E = L), private beta copies = beta0; trust radii
// reset to 1 unless keep_trust.
int launch_init_state(const DevLayout &d, const double *beta0_dev, int threads, void *stream,
                      bool keep_trust = false);
// E32 = (float) E on every shard.
int launch_e_to_f32(const DevLayout &d, int threads, void *stream);
// Build the row -> columns index (row_ptr, row_col) from the column slices.  scratch: K int32
// counts + K int64 fill cursors + (K / 8192 + 2) int64 block sums.
int launch_build_row_index(const DevLayout &d, int64_t *row_ptr, int32_t *row_col, int32_t *cnt, int64_t *cursor,
                           int64_t *block_sums, void *stream);
size_t row_index_scan_blocks(int64_t K);
// Diagnostic: the coordinate step's e^x and CUDA's exp on n device values.
int launch_exp_selftest(const double *x, long long n, double *ours, double *ref, void *stream);
int launch_div_selftest(const double *a, const double *b, long long n, double *ours, double *ref, void *stream);
// Weighted counts of a fit with subject weights w_kept (device [N]): nev_w[i] = w_i n_i and
// ytx_w[j] = sum over X_j's (subject, y) pairs of w_i y, both exact (integer sums).
int launch_weighted_counts(const DevLayout &d, const int32_t *w_kept, int32_t *nev_w, double *ytx_w, void *stream);
int launch_fit(const DevLayout &d, const FitParams &p, FitOut *out_dev, double *hist_dev,
               int threads, void *stream, bool fp32 = false);
int launch_grad_hess(const DevLayout &d, int32_t j, const FitParams &p, FitOut *out_dev,
                     int threads, void *stream);
// The gradient kernel on only `ctas` of the S CTAs the all-reduce counts (a wait-bound test).
int launch_grad_hess_partial(const DevLayout &d, int32_t j, const FitParams &p, FitOut *out_dev,
                             int threads, int ctas, void *stream);
int fit_kernel_max_blocks_per_sm(int threads, int *blocks);
// Clusters of `cluster` CTAs of the FP64 fit kernel that can be resident at once (0 if none).
int fit_kernel_max_clusters(int threads, int cluster, int *clusters);
// Independent fits in one cooperative launch: CTA b runs shard map[b].y of fit map[b].x
// (entries and map in device memory; every fit's CTAs form its own all-reduce team).
// The batched fits in one persistent cooperative launch of `ctas` CTAs.  entries (device) are
// in scheduling order; team_start (device, n + 1) is the prefix sum of the entries' team sizes;
// counters (device, 1 + n unsigned, zeroed by launch_batch_prep) hold the ticket counter and
// one arrival count per fit.  A CTA takes tickets in order: ticket t is shard
// t - team_start[f] of the fit f whose range holds t.  The fit starts when its whole team has
// arrived (a wait bounded by assemble_ns) and computes exactly what it computes alone.
int launch_fit_queue(const BatchEntry *entries_dev, const int *team_start_dev, int n, unsigned *counters_dev,
                     int ctas, int threads, void *stream, int mode, long long assemble_ns);
// Zero the ticket/arrival counters and every entry's out / out32 (one small launch).
int launch_batch_prep(const BatchEntry *entries_dev, int n, unsigned *counters_dev, void *stream);
// Gather every fit's out, out32 and beta (shard 0's copy) into one buffer: outs[n], outs32[n],
// then the betas at beta_off[f] doubles from `betas`.
int launch_batch_gather(const BatchEntry *entries_dev, int n, FitOut *outs, FitOut *outs32, double *betas,
                        const long long *beta_off_dev, void *stream);

// What the serving layer needs of a dataset handle: its device, block size and layout (whose
// static arrays it shares; the state pointers it replaces with a fit slot's own).
struct HandleView {
    int device;
    int threads;
    DevLayout d;
    const int64_t *kept_from;  // host [N]: input subject index of each kept subject
    const int32_t *nev_host;   // host [N]: n_i
    int64_t subjects_in;
    int32_t max_nev;           // largest n_i
};

// Subject weights given per input subject -> per kept subject (host arrays).  SCCS_E_INVAL for
// a negative weight or a product w_i n_i above 2^31 - 1 (the message names the subject).
int map_subject_weights(const HandleView &v, const int32_t *w_in, int32_t *w_kept);

}  // namespace sccs

struct sccs_handle;
// Fill `v` from a created handle; false if h is null.
bool sccs_handle_view(const sccs_handle *h, sccs::HandleView *v);

// Record a thread-local error message for sccs_last_error and return `code`.
extern "C" int sccs_set_error(int code, const char *msg);
