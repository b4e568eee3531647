// Create-time layout built on the device: the stages that touch every row and every nonzero
// (kept subjects and rows, each column's kept rows and subjects, Y'X_j, the
// per-column event pairs, the subject segments and the jagged-diagonal slices of a shard
// partition, the marks of the narrow columns).  The host keeps the decisions over columns
// (which columns are narrow or cluster columns, how they are grouped), made from the per-column
// counts these stages return.  Internal header.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace sccs {
namespace lay {

// flags[] words written by the layout kernels
enum Flag : int {
    kFBigN = 0,        // 1 when some n_i >= 2^31
    kFDup,             // smallest column with a repeated kept row (kNone: none)
    kFUnsorted,        // 1 when some column's rows are not ascending
    kFMaxSeg,          // largest slice: segments (at least 1)
    kFMaxRows,         //                nonzeros (at least 1)
    kFLmax,            // longest subject segment of any column
    kFCount
};
constexpr unsigned long long kNone = ~0ull;

// Scratch device memory of one build, from a stream-ordered pool that the library keeps for the
// life of the process (so a later build reuses the pages instead of mapping them again).
class Scratch {
public:
    explicit Scratch(cudaStream_t st) : st_(st) {}
    ~Scratch() { release(); }
    void *get(size_t bytes);          // null on failure
    void release();                   // every block back to the pool (stream-ordered)
    template <class T>
    T *get_n(size_t n) {
        return static_cast<T *>(get(sizeof(T) * (n > 0 ? n : 1)));
    }

private:
    cudaStream_t st_;
    std::vector<void *> blocks_;
};

// An exclusive scan split in two: count() sums the chunks and returns the total (one small
// device-to-host copy), apply() hands every element its prefix.
struct ScanBuf {
    long long *chunks = nullptr;   // per chunk of the input, its exclusive offset
    long long nch = 0;
    long long n = 0;
};

// Everything the stages share.  Device pointers unless noted.
struct Ctx {
    cudaStream_t st = nullptr;
    Scratch *scr = nullptr;
    int64_t K = 0, nnz_in = 0;
    int32_t J = 0;
    // inputs, as given
    const int64_t *pid = nullptr;
    const int32_t *y = nullptr;
    const double *L = nullptr;
    const int64_t *col_ptr = nullptr;
    const int32_t *ri = nullptr;
    unsigned long long *flags = nullptr;     // kFCount
    unsigned long long *flags_h = nullptr;   // pinned host copy
    long long *total_d = nullptr;            // a scan total
    long long *total_h = nullptr;            // pinned
    // subjects
    int64_t nsub = 0, Nk = 0, Kk = 0;
    int64_t *subidx = nullptr;     // K: input subject of each input row
    int64_t *sub_start = nullptr;  // nsub+1
    int64_t *sub_n = nullptr;      // nsub: n_i
    int64_t *sub_new = nullptr;    // nsub: kept index, or -1
    ScanBuf rows_sb;               // the kept rows' scan over subjects (count, then fill)
    int32_t *newrow = nullptr;     // K: kept row of each input row, -1 if dropped (only when rows are dropped)
    int32_t *ksub = nullptr;       // Kk: kept subject of each kept row
    int32_t *ky = nullptr;         // Kk: its event count
    // columns
    int64_t nnz = 0;
    int64_t *cptr = nullptr;       // J+1
    int32_t *crow = nullptr;       // nnz: each column's kept rows, ascending
    int32_t *csub = nullptr;       // nnz: their subjects
    int32_t *cy = nullptr;         // nnz: their event counts
    // column segments: the runs of one subject in a column (in column order, subjects ascending)
    int64_t nseg = 0;
    int64_t *cs_start = nullptr;   // nseg+1: first nonzero
    int32_t *cs_sub = nullptr;     // nseg
    int32_t *cs_len = nullptr;     // nseg
    int32_t *cs_y = nullptr;       // nseg: sum of y over the segment's rows
    int64_t *cseg_ptr = nullptr;   // J+1: each column's first segment
    int32_t lmax = 0;
};

// A partition of the kept subjects into Sp shards and its (shard, column) slices over the columns
// with mask[j] (every column when mask is null).
struct SliceSet {
    int32_t Sp = 0;
    const int64_t *shard_pat = nullptr;   // Sp+1 (device)
    const uint8_t *mask = nullptr;        // J (device) or null
    int64_t *sl_a = nullptr;              // Sp*(J+1): first column segment of the slice
    int64_t *sl_nnz = nullptr;            // Sp*(J+1)
    int64_t *sl_nseg = nullptr;           // Sp*(J+1)
    ScanBuf sc_row, sc_seg, sc_grp;
    int64_t tr = 0, ts = 0, tg = 0;       // totals: nonzeros, segments, groups
    int64_t max_seg = 1, max_rows = 1;
};

// Stages, in order, on inputs the host has validated.  Each returns 0 or a cudaError_t value;
// what the caller reports as bad input (n_i too large, a duplicate row) is left in flags_h.
int upload_inputs(Ctx &c, const int64_t *pid, const int32_t *y, const double *L, const int64_t *col_ptr,
                  const int32_t *row_idx);
int subjects_count(Ctx &c);                                         // nsub, Nk, Kk; flags_h[kFBigN]
int subjects_fill(Ctx &c, int64_t *pat_ptr, int32_t *nev, int64_t *kept_from, double *Lk);
int columns(Ctx &c, std::vector<int64_t> &cptr_h, std::vector<int64_t> &ytx_h);   // flags_h[kFDup]
int segments(Ctx &c, std::vector<int64_t> &cseg_ptr_h);
int pairs_count(Ctx &c, ScanBuf &sb, int64_t &npairs);
int pairs_fill(Ctx &c, ScanBuf &sb, int64_t npairs, int32_t *ysub, int32_t *ycnt, std::vector<int64_t> &ycol_ptr_h);
int shards(Ctx &c, const int64_t *pat_ptr, int32_t Sp, int64_t *shard_pat, int64_t *shard_row);
// nnz_h / nseg_h (optional): the slice counts on the host, shard-major
int slices_count(Ctx &c, SliceSet &ss, std::vector<int64_t> *nnz_h, std::vector<int64_t> *nseg_h);
int slices_fill(Ctx &c, SliceSet &ss, int64_t *slice_row, int64_t *slice_seg, int64_t *slice_grp, int32_t *rows,
                int2 *segs, int64_t *grp_base);
// lp[j] for each listed column: the largest column j' < j holding one of j's subjects (-1: none)
int last_prev_columns(Ctx &c, const int64_t *pat_ptr, const int64_t *row_ptr, const int32_t *row_col,
                      const std::vector<int32_t> &cols, std::vector<int32_t> &lp);
// Narrow columns' segments and rows.  Per listed column j: nar_first (its first segment in
// nar_seg), row_first (its first row in nar_row), and for the marks: run_wide (the wide column
// before its run when its group starts the run, else -1), prev0 / prevm (the previous group's
// first column and size when its group does not start the run, else prevm = 0).
struct NarrowCol {
    int32_t j, run_wide, prev0, prevm;
    int64_t nar_first, row_first;
};
int narrow_fill(Ctx &c, const int64_t *pat_ptr, const int64_t *row_ptr, const int32_t *row_col,
                const std::vector<NarrowCol> &cols, int4 *nar_seg, int32_t *nar_row, int32_t after_wide);

}  // namespace lay
}  // namespace sccs
