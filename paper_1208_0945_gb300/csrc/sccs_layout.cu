// Create-time layout on the device (see sccs_layout.h).  Every stage is a few grid-stride
// kernels or an exclusive scan over rows, nonzeros, subjects, segments or slices; a stage ends
// with a small device-to-host copy only where the host needs a count to size the next arrays.
// The results are the layout the fit kernels read (Section 2.4's representation of M and X_j,
// in the sharded jagged-diagonal form described in sccs_kernels.cu), element for element.
#include "sccs_layout.h"

#include <algorithm>
#include <cstring>
#include <mutex>

#include "sccs_internal.h"

namespace sccs {
namespace lay {
namespace {

constexpr int kTB = 256;                       // threads of every layout block
constexpr int kRounds = 16;                    // rows of kTB elements per scan chunk
constexpr long long kChunk = static_cast<long long>(kTB) * kRounds;
constexpr unsigned kAll = 0xffffffffu;
constexpr int kBins = 512;                     // per-warp length bins in shared memory
constexpr int kWarpsPB = kTB / 32;

int grid_for(long long n, int per = kTB) {
    const long long b = (n + per - 1) / per;
    return static_cast<int>(std::max<long long>(1, std::min<long long>(b, 152LL * 64)));
}

// ------------------------------------------------------------------ helpers

// The column (or segment list) holding element e: the largest c with ptr[c] <= e (ptr[0..n],
// ascending; with empty entries the one whose range actually holds e).
__device__ __forceinline__ int owner_of(const long long *ptr, int n, long long e) {
    int lo = 0, hi = n;                        // invariant: ptr[lo] <= e < ptr[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (ptr[mid] <= e) lo = mid;
        else hi = mid;
    }
    return lo;
}

// First index in a[lo, hi) with a[i] >= v.
template <class T>
__device__ __forceinline__ long long lower_bound_dev(const T *a, long long lo, long long hi, long long v) {
    while (lo < hi) {
        const long long mid = lo + ((hi - lo) >> 1);
        if (static_cast<long long>(a[mid]) < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Does subject x have a row in column j?  (each row's columns are ascending)
__device__ bool subject_has_column(const long long *pat_ptr, const long long *row_ptr, const int *row_col, int x,
                                   int j) {
    for (long long k = pat_ptr[x]; k < pat_ptr[x + 1]; ++k) {
        const long long a = row_ptr[k], b = row_ptr[k + 1];
        const long long q = lower_bound_dev(row_col, a, b, j);
        if (q < b && row_col[q] == j) return true;
    }
    return false;
}

__device__ __forceinline__ long long block_excl_scan(long long v, long long &total, long long *wt) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(kAll, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) wt[w] = x;
    __syncthreads();
    if (w == 0) {
        long long t = lane < kWarpsPB ? wt[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long u = __shfl_up_sync(kAll, t, o);
            if (lane >= o) t += u;
        }
        if (lane < kWarpsPB) wt[lane] = t;
    }
    __syncthreads();
    const long long before = w > 0 ? wt[w - 1] : 0;
    total = wt[kWarpsPB - 1];
    __syncthreads();
    return before + x - v;
}

// ------------------------------------------------------------------ scans

template <class F>
__global__ void __launch_bounds__(kTB) scan_totals_kernel(F f, long long n, long long *chunks) {
    __shared__ long long wt[kWarpsPB];
    const long long base = static_cast<long long>(blockIdx.x) * kChunk;
    long long s = 0;
    for (int r = 0; r < kRounds; ++r) {
        const long long i = base + static_cast<long long>(r) * kTB + threadIdx.x;
        if (i < n) s += f(i);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(kAll, s, o);
    if ((threadIdx.x & 31) == 0) wt[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int q = 0; q < kWarpsPB; ++q) t += wt[q];
        chunks[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kTB) scan_offsets_kernel(long long *chunks, long long nch, long long *total) {
    __shared__ long long wt[kWarpsPB];
    long long run = 0;
    for (long long b = 0; b < nch; b += kTB) {
        const long long i = b + threadIdx.x;
        const long long v = i < nch ? chunks[i] : 0;
        long long t;
        const long long ex = block_excl_scan(v, t, wt);
        if (i < nch) chunks[i] = run + ex;
        run += t;
    }
    if (threadIdx.x == 0) *total = run;
}

template <class F, class G>
__global__ void __launch_bounds__(kTB) scan_apply_kernel(F f, G g, long long n, const long long *chunks) {
    __shared__ long long wt[kWarpsPB];
    const long long base = static_cast<long long>(blockIdx.x) * kChunk;
    long long run = chunks[blockIdx.x];
    for (int r = 0; r < kRounds; ++r) {
        if (base + static_cast<long long>(r) * kTB >= n) break;   // block-uniform
        const long long i = base + static_cast<long long>(r) * kTB + threadIdx.x;
        const long long v = i < n ? f(i) : 0;
        long long t;
        const long long ex = block_excl_scan(v, t, wt);
        if (i < n) g(i, run + ex, v);
        run += t;
    }
}

// count(): the scan's total (synchronous); the chunk offsets stay in sb for apply()
template <class F>
int scan_count(Ctx &c, ScanBuf &sb, F f, long long n, long long &total) {
    sb.n = n;
    sb.nch = (n + kChunk - 1) / kChunk;
    if (sb.nch == 0) {
        total = 0;
        return 0;
    }
    sb.chunks = c.scr->get_n<long long>(static_cast<size_t>(sb.nch));
    if (!sb.chunks) return static_cast<int>(cudaErrorMemoryAllocation);
    scan_totals_kernel<<<static_cast<unsigned>(sb.nch), kTB, 0, c.st>>>(f, n, sb.chunks);
    scan_offsets_kernel<<<1, kTB, 0, c.st>>>(sb.chunks, sb.nch, c.total_d);
    cudaError_t e = cudaMemcpyAsync(c.total_h, c.total_d, sizeof(long long), cudaMemcpyDeviceToHost, c.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
    if (e != cudaSuccess) return static_cast<int>(e);
    total = *c.total_h;
    return 0;
}

template <class F, class G>
int scan_apply(Ctx &c, const ScanBuf &sb, F f, G g) {
    if (sb.nch == 0) return 0;
    scan_apply_kernel<<<static_cast<unsigned>(sb.nch), kTB, 0, c.st>>>(f, g, sb.n, sb.chunks);
    return static_cast<int>(cudaGetLastError());
}

// ------------------------------------------------------------------ flags

__global__ void flags_init_kernel(unsigned long long *flags) {
    const int t = threadIdx.x;
    if (t < kFCount) {
        flags[t] = t == kFDup ? kNone : (t == kFMaxSeg || t == kFMaxRows ? 1ull : 0ull);
    }
}

// ------------------------------------------------------------------ subjects

struct HeadF {
    const long long *pid;
    __device__ long long operator()(long long i) const { return (i == 0 || pid[i] != pid[i - 1]) ? 1 : 0; }
};
struct HeadG {
    long long *sub_start, *subidx;
    __device__ void operator()(long long i, long long pre, long long v) const {
        if (v) sub_start[pre] = i;
        subidx[i] = pre + v - 1;
    }
};

__global__ void subject_n_kernel(long long nsub, const long long *sub_start, const int *y, long long *sub_n,
                                 unsigned long long *flags) {
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < nsub;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        long long n = 0;
        for (long long k = sub_start[i]; k < sub_start[i + 1]; ++k) n += y[k];
        sub_n[i] = n;
        if (n >= (1ll << 31)) flags[kFBigN] = 1;
    }
}

struct KeepF {
    const long long *sub_n;
    __device__ long long operator()(long long i) const { return sub_n[i] > 0 ? 1 : 0; }
};
struct KeepG {
    long long *sub_new;
    __device__ void operator()(long long i, long long pre, long long v) const { sub_new[i] = v ? pre : -1; }
};
struct RowsF {
    const long long *sub_n, *sub_start;
    __device__ long long operator()(long long i) const { return sub_n[i] > 0 ? sub_start[i + 1] - sub_start[i] : 0; }
};
struct RowsG {
    const long long *sub_n, *sub_new;
    long long *pat_ptr, *kept_from;
    int *nev;
    __device__ void operator()(long long i, long long pre, long long) const {
        if (sub_n[i] <= 0) return;
        const long long q = sub_new[i];
        pat_ptr[q] = pre;
        nev[q] = static_cast<int>(sub_n[i]);
        kept_from[q] = i;
    }
};

__global__ void put_i64_kernel(long long *p, long long v) { *p = v; }

__global__ void kept_rows_kernel(long long K, const long long *subidx, const long long *sub_start,
                                 const long long *sub_new, const long long *pat_ptr, const int *y, const double *L,
                                 int *newrow, int *ksub, int *ky, double *Lk) {
    for (long long k = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; k < K;
         k += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long i = subidx[k];
        const long long q = sub_new[i];
        if (q < 0) {
            if (newrow) newrow[k] = -1;
            continue;
        }
        const long long kr = pat_ptr[q] + (k - sub_start[i]);
        if (newrow) newrow[k] = static_cast<int>(kr);
        Lk[kr] = L[k];
        ksub[kr] = static_cast<int>(q);
        ky[kr] = y[k];
    }
}

// ------------------------------------------------------------------ columns

struct KeepNzF {
    const int *ri, *newrow;
    __device__ long long operator()(long long e) const { return newrow[ri[e]] >= 0 ? 1 : 0; }
};
struct KeepNzG {
    const int *ri, *newrow;
    const long long *col_ptr;
    int J;
    int *crow;
    long long *cptr;
    __device__ void operator()(long long e, long long pre, long long v) const {
        if (v) crow[pre] = newrow[ri[e]];
        const int j = owner_of(col_ptr, J, e);
        if (col_ptr[j] == e) cptr[j] = pre;     // empty columns are filled in on the host
    }
};

__global__ void column_check_kernel(long long nnz, int J, const long long *cptr, const int *crow, uint8_t *unsorted,
                                    unsigned long long *flags) {
    for (long long e = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; e < nnz;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int j = owner_of(cptr, J, e);
        if (e == cptr[j]) continue;
        const int a = crow[e - 1], b = crow[e];
        if (b < a) {
            unsorted[j] = 1;
            flags[kFUnsorted] = 1;
        } else if (b == a) {
            atomicMin(&flags[kFDup], static_cast<unsigned long long>(j));
        }
    }
}

// csub / cy by one random lookup per nonzero; Y'X_j by runs of one column within a warp
__global__ void column_lookup_kernel(long long nnz, int J, const long long *cptr, const int *crow, const int *ksub,
                                     const int *ky, int *csub, int *cy, unsigned long long *ytx) {
    const int lane = threadIdx.x & 31;
    const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
    for (long long e0 = static_cast<long long>(blockIdx.x) * blockDim.x; e0 < nnz; e0 += stride) {
        const long long e = e0 + threadIdx.x;
        const bool act = e < nnz;
        int j = -1;
        long long v = 0;
        if (act) {
            const int r = crow[e];
            csub[e] = ksub[r];
            const int yv = ky[r];
            cy[e] = yv;
            v = yv;
            j = owner_of(cptr, J, e);
        }
        // inclusive segmented sum over lanes of the same column (a column's lanes are adjacent)
        long long s = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(kAll, s, o);
            const int jt = __shfl_up_sync(kAll, j, o);
            if (lane >= o && jt == j) s += t;
        }
        const int jn = __shfl_down_sync(kAll, j, 1);
        const bool last = lane == 31 || jn != j;
        if (act && last && s != 0) atomicAdd(&ytx[j], static_cast<unsigned long long>(s));
    }
}

struct SegHeadF {
    const long long *cptr;
    const int *csub;
    int J;
    __device__ long long operator()(long long e) const {
        const int j = owner_of(cptr, J, e);
        return (e == cptr[j] || csub[e] != csub[e - 1]) ? 1 : 0;
    }
};
struct SegHeadG {
    const long long *cptr;
    const int *csub;
    int J;
    long long *cs_start, *cseg_first;
    int *cs_sub;
    __device__ void operator()(long long e, long long pre, long long v) const {
        if (!v) return;
        cs_start[pre] = e;
        cs_sub[pre] = csub[e];
        const int j = owner_of(cptr, J, e);
        if (e == cptr[j]) cseg_first[j] = pre;
    }
};

__global__ void segment_values_kernel(long long nseg, const long long *cs_start, const int *cy, int *cs_len, int *cs_y,
                                      unsigned long long *flags) {
    int lm = 0;
    for (long long s = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; s < nseg;
         s += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long a = cs_start[s], b = cs_start[s + 1];
        long long t = 0;
        for (long long e = a; e < b; ++e) t += cy[e];
        cs_len[s] = static_cast<int>(b - a);
        cs_y[s] = static_cast<int>(t);
        lm = max(lm, static_cast<int>(b - a));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) lm = max(lm, __shfl_xor_sync(kAll, lm, o));
    if ((threadIdx.x & 31) == 0 && lm > 0) atomicMax(&flags[kFLmax], static_cast<unsigned long long>(lm));
}

struct PairF {
    const int *cs_y;
    __device__ long long operator()(long long s) const { return cs_y[s] > 0 ? 1 : 0; }
};
struct PairG {
    const int *cs_y, *cs_sub;
    const long long *cseg_ptr;
    int J;
    int *ysub, *ycnt;
    long long *ycol_first;
    __device__ void operator()(long long s, long long pre, long long v) const {
        const int j = owner_of(cseg_ptr, J, s);
        if (s == cseg_ptr[j]) ycol_first[j] = pre;
        if (v) {
            ysub[pre] = cs_sub[s];
            ycnt[pre] = cs_y[s];
        }
    }
};

// ------------------------------------------------------------------ shards and slices

// Shards at subject boundaries, balanced by rows (one thread: Sp binary searches)
// Shard s starts at the first subject whose rows begin at or after K s / Sp (one thread per shard:
// the targets rise with s, so the starts do too).
__global__ void shards_kernel(const long long *pat_ptr, long long Nk, long long Kk, int Sp, long long *shard_pat,
                              long long *shard_row) {
    for (int s = static_cast<int>(blockIdx.x * blockDim.x + threadIdx.x); s <= Sp;
         s += static_cast<int>(gridDim.x * blockDim.x)) {
        long long p = 0;
        if (s == Sp) p = Nk;
        else if (s > 0) p = min(lower_bound_dev(pat_ptr, 0, Nk + 1, (Kk * s) / Sp), Nk);
        shard_pat[s] = p;
        shard_row[s] = pat_ptr[p];
    }
}

__global__ void slice_count_kernel(int Sp, int J, const long long *shard_pat, const uint8_t *mask,
                                   const long long *cseg_ptr, const int *cs_sub, const long long *cs_start,
                                   long long *sl_a, long long *sl_nnz, long long *sl_nseg, unsigned long long *flags) {
    const long long n = static_cast<long long>(Sp) * (J + 1);
    for (long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; idx < n;
         idx += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int s = static_cast<int>(idx / (J + 1)), j = static_cast<int>(idx % (J + 1));
        long long a = 0, ns = 0, nz = 0;
        if (j < J && (!mask || mask[j])) {
            const long long lo = cseg_ptr[j], hi = cseg_ptr[j + 1];
            a = lower_bound_dev(cs_sub, lo, hi, shard_pat[s]);
            const long long b = lower_bound_dev(cs_sub, a, hi, shard_pat[s + 1]);
            ns = b - a;
            nz = cs_start[b] - cs_start[a];
            if (ns > 1) atomicMax(&flags[kFMaxSeg], static_cast<unsigned long long>(ns));
            if (nz > 1) atomicMax(&flags[kFMaxRows], static_cast<unsigned long long>(nz));
        }
        sl_a[idx] = a;
        sl_nnz[idx] = nz;
        sl_nseg[idx] = ns;
    }
}

struct ArrF {
    const long long *a;
    __device__ long long operator()(long long i) const { return a[i]; }
};
struct GrpF {
    const long long *nseg;
    __device__ long long operator()(long long i) const { return (nseg[i] + 31) / 32; }
};
struct PutG {
    long long *out;
    __device__ void operator()(long long i, long long pre, long long) const { out[i] = pre; }
};

// One warp per slice: its segments longest first, ties in column order (subject order), by a
// stable counting sort over the lengths.
__global__ void __launch_bounds__(kTB) slice_sort_kernel(long long nsl, int J, const long long *sl_a,
                                                          const long long *slice_seg, const int *cs_len,
                                                          const int *cs_sub, int2 *segs, long long *sorted_seg,
                                                          int *gbins, long long gstride, bool use_smem) {
    __shared__ int sbins[kWarpsPB][kBins];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long gw = static_cast<long long>(blockIdx.x) * kWarpsPB + w;
    const long long nw = static_cast<long long>(gridDim.x) * kWarpsPB;
    int *bins = use_smem ? sbins[w] : gbins + gw * gstride;
    const unsigned lt = (1u << lane) - 1u;
    for (long long sl = gw; sl < nsl; sl += nw) {
        if (sl % (J + 1) == J) continue;
        const long long spos = slice_seg[sl], n = slice_seg[sl + 1] - spos;
        if (n == 0) continue;
        const long long a0 = sl_a[sl];
        int ml = 0;
        for (long long q = lane; q < n; q += 32) ml = max(ml, cs_len[a0 + q]);
#pragma unroll
        for (int o = 16; o; o >>= 1) ml = max(ml, __shfl_xor_sync(kAll, ml, o));
        for (int l = lane; l <= ml; l += 32) bins[l] = 0;
        __syncwarp();
        for (long long q0 = 0; q0 < n; q0 += 32) {
            const long long q = q0 + lane;
            const bool act = q < n;
            const int len = act ? cs_len[a0 + q] : -1;
            const unsigned m = __match_any_sync(kAll, len);
            if (act && lane == __ffs(m) - 1) bins[len] += __popc(m);
            __syncwarp();
        }
        // bins[l] <- segments longer than l (the first position of length l)
        long long run = 0;
        for (int top = ml; top >= 1; top -= 32) {
            const int l = top - lane;
            const int h = l >= 1 ? bins[l] : 0;
            int x = h;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(kAll, x, o);
                if (lane >= o) x += t;
            }
            __syncwarp();
            if (l >= 1) bins[l] = static_cast<int>(run + x - h);
            run += __shfl_sync(kAll, x, 31);
        }
        __syncwarp();
        for (long long q0 = 0; q0 < n; q0 += 32) {
            const long long q = q0 + lane;
            const bool act = q < n;
            const int len = act ? cs_len[a0 + q] : -1;
            const unsigned m = __match_any_sync(kAll, len);
            const int base = act ? bins[len] : 0;
            __syncwarp();
            if (act && lane == __ffs(m) - 1) bins[len] = base + __popc(m);
            __syncwarp();
            if (act) {
                const long long pos = spos + base + __popc(m & lt);
                segs[pos] = make_int2(cs_sub[a0 + q], len);
                sorted_seg[pos] = a0 + q;
            }
        }
        __syncwarp();
    }
}

__device__ __forceinline__ long long slice_of_group(const long long *slice_grp, long long nsl, long long g) {
    long long lo = 0, hi = nsl;                 // last sl with slice_grp[sl] <= g
    while (hi - lo > 1) {
        const long long mid = lo + ((hi - lo) >> 1);
        if (slice_grp[mid] <= g) lo = mid;
        else hi = mid;
    }
    return lo;
}

// One warp per 32-segment group: its rows.
__global__ void __launch_bounds__(kTB) group_rows_kernel(long long tg, long long nsl, const long long *slice_grp,
                                                          const long long *slice_seg, const int2 *segs,
                                                          long long *grp_rows) {
    const int lane = threadIdx.x & 31;
    const long long nw = static_cast<long long>(gridDim.x) * kWarpsPB;
    for (long long g = static_cast<long long>(blockIdx.x) * kWarpsPB + (threadIdx.x >> 5); g < tg; g += nw) {
        const long long sl = slice_of_group(slice_grp, nsl, g);
        const long long s0 = slice_seg[sl] + 32 * (g - slice_grp[sl]), s1 = slice_seg[sl + 1];
        int v = s0 + lane < s1 ? segs[s0 + lane].y : 0;
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kAll, v, o);
        if (lane == 0) grp_rows[g] = v;
    }
}

// One warp per group: its rows diagonal by diagonal (segments longest first, so the lanes with a
// row on diagonal t are a prefix of the group).
__global__ void __launch_bounds__(kTB) jds_fill_kernel(long long tg, long long nsl, const long long *slice_grp,
                                                        const long long *slice_seg, const int2 *segs,
                                                        const long long *sorted_seg, const long long *cs_start,
                                                        const long long *grp_base, const int *crow, int *rows) {
    const int lane = threadIdx.x & 31;
    const long long nw = static_cast<long long>(gridDim.x) * kWarpsPB;
    for (long long g = static_cast<long long>(blockIdx.x) * kWarpsPB + (threadIdx.x >> 5); g < tg; g += nw) {
        const long long sl = slice_of_group(slice_grp, nsl, g);
        const long long s0 = slice_seg[sl] + 32 * (g - slice_grp[sl]), s1 = slice_seg[sl + 1];
        const bool valid = s0 + lane < s1;
        const int len = valid ? segs[s0 + lane].y : 0;
        const long long start = valid ? cs_start[sorted_seg[s0 + lane]] : 0;
        const int maxlen = __shfl_sync(kAll, len, 0);
        long long base = grp_base[g];
        for (int t = 0; t < maxlen; ++t) {
            const bool act = len > t;
            const unsigned m = __ballot_sync(kAll, act);
            if (act) rows[base + lane] = crow[start + t];
            base += __popc(m);
        }
    }
}

// ------------------------------------------------------------------ column groups and narrow columns

// One block per listed column j: the largest column before j holding one of j's subjects.
__global__ void __launch_bounds__(kTB) last_prev_kernel(const int *cols, int ncols, const long long *cptr,
                                                         const int *csub, const long long *pat_ptr,
                                                         const long long *row_ptr, const int *row_col, int *lp) {
    __shared__ int wbest[kWarpsPB];
    for (int b = blockIdx.x; b < ncols; b += gridDim.x) {
        const int j = cols[b];
        int best = -1;
        for (long long e = cptr[j] + threadIdx.x; e < cptr[j + 1]; e += blockDim.x) {
            const int x = csub[e];
            for (long long k = pat_ptr[x]; k < pat_ptr[x + 1]; ++k) {
                const long long a = row_ptr[k], q = lower_bound_dev(row_col, a, row_ptr[k + 1], j);
                if (q > a) best = max(best, row_col[q - 1]);
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) best = max(best, __shfl_xor_sync(kAll, best, o));
        if ((threadIdx.x & 31) == 0) wbest[threadIdx.x >> 5] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = -1;
            for (int q = 0; q < kWarpsPB; ++q) t = max(t, wbest[q]);
            lp[b] = t;
        }
        __syncthreads();
    }
}

struct NarrowColDev {
    int j, run_wide, prev0, prevm;
    long long nar_first, row_first;
};

__global__ void __launch_bounds__(kTB) narrow_fill_kernel(const NarrowColDev *cols, int ncols, const long long *cptr,
                                                           const long long *cseg_ptr, const long long *cs_start,
                                                           const int *cs_sub, const int *cs_len, const int *crow,
                                                           const long long *pat_ptr, const long long *row_ptr,
                                                           const int *row_col, int4 *nar_seg, int *nar_row,
                                                           int after_wide) {
    for (int b = blockIdx.x; b < ncols; b += gridDim.x) {
        const NarrowColDev nc = cols[b];
        const long long c0 = cptr[nc.j], c1 = cptr[nc.j + 1];
        for (long long e = c0 + threadIdx.x; e < c1; e += blockDim.x) nar_row[nc.row_first + (e - c0)] = crow[e];
        const long long q0 = cseg_ptr[nc.j], q1 = cseg_ptr[nc.j + 1];
        for (long long q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
            const int x = cs_sub[q];
            int w = 0;
            if (nc.run_wide >= 0) {
                if (subject_has_column(pat_ptr, row_ptr, row_col, x, nc.run_wide)) w = after_wide;
            } else {
                for (int c = 0; c < nc.prevm; ++c)
                    if (subject_has_column(pat_ptr, row_ptr, row_col, x, nc.prev0 + c)) {
                        w = c + 1;
                        break;
                    }
            }
            nar_seg[nc.nar_first + (q - q0)] =
                make_int4(x, cs_len[q], static_cast<int>(nc.row_first + (cs_start[q] - c0)), w);
        }
    }
}

// ------------------------------------------------------------------ the scratch pool

std::mutex g_pool_mu;
cudaMemPool_t g_pool[64] = {};

cudaMemPool_t pool_for_current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        // keep up to 8 GB mapped between builds
        unsigned long long keep = 8ull << 30;
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pool[dev] = p;
    }
    return g_pool[dev];
}

}  // namespace

// ------------------------------------------------------------------ Scratch

void *Scratch::get(size_t bytes) {
    cudaMemPool_t p = pool_for_current_device();
    if (!p) return nullptr;
    void *ptr = nullptr;
    if (cudaMallocFromPoolAsync(&ptr, std::max<size_t>(bytes, 16), p, st_) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    blocks_.push_back(ptr);
    return ptr;
}

void Scratch::release() {
    for (void *b : blocks_) cudaFreeAsync(b, st_);
    blocks_.clear();
}

// ------------------------------------------------------------------ stages

int upload_inputs(Ctx &c, const int64_t *pid, const int32_t *y, const double *L, const int64_t *col_ptr,
                  const int32_t *row_idx) {
    const size_t K = static_cast<size_t>(c.K), nz = static_cast<size_t>(c.nnz_in), J1 = static_cast<size_t>(c.J) + 1;
    int64_t *dpid = c.scr->get_n<int64_t>(K);
    int32_t *dy = c.scr->get_n<int32_t>(K);
    double *dL = c.scr->get_n<double>(K);
    int64_t *dcp = c.scr->get_n<int64_t>(J1);
    int32_t *dri = c.scr->get_n<int32_t>(nz);
    c.flags = c.scr->get_n<unsigned long long>(kFCount);
    c.total_d = c.scr->get_n<long long>(1);
    if (!dpid || !dy || !dL || !dcp || !dri || !c.flags || !c.total_d)
        return static_cast<int>(cudaErrorMemoryAllocation);
    cudaError_t e = cudaSuccess;
    if (K) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(dpid, pid, 8 * K, cudaMemcpyHostToDevice, c.st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dy, y, 4 * K, cudaMemcpyHostToDevice, c.st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dL, L, 8 * K, cudaMemcpyHostToDevice, c.st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(dcp, col_ptr, 8 * J1, cudaMemcpyHostToDevice, c.st);
    if (nz) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(dri, row_idx, 4 * nz, cudaMemcpyHostToDevice, c.st);
    }
    if (e != cudaSuccess) return static_cast<int>(e);
    c.pid = dpid;
    c.y = dy;
    c.L = dL;
    c.col_ptr = dcp;
    c.ri = dri;
    flags_init_kernel<<<1, 32, 0, c.st>>>(c.flags);
    return static_cast<int>(cudaGetLastError());
}

static int read_flags(Ctx &c) {
    cudaError_t e = cudaMemcpyAsync(c.flags_h, c.flags, sizeof(unsigned long long) * kFCount, cudaMemcpyDeviceToHost,
                                    c.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
    return static_cast<int>(e);
}

int subjects_count(Ctx &c) {
    const long long *pid = reinterpret_cast<const long long *>(c.pid);
    ScanBuf sb;
    long long nsub = 0;
    int rc = scan_count(c, sb, HeadF{pid}, c.K, nsub);
    if (rc) return rc;
    c.nsub = nsub;
    c.subidx = c.scr->get_n<int64_t>(static_cast<size_t>(c.K));
    c.sub_start = c.scr->get_n<int64_t>(static_cast<size_t>(nsub) + 1);
    c.sub_n = c.scr->get_n<int64_t>(static_cast<size_t>(nsub));
    c.sub_new = c.scr->get_n<int64_t>(static_cast<size_t>(nsub));
    if (!c.subidx || !c.sub_start || !c.sub_n || !c.sub_new) return static_cast<int>(cudaErrorMemoryAllocation);
    long long *ss = reinterpret_cast<long long *>(c.sub_start);
    if ((rc = scan_apply(c, sb, HeadF{pid}, HeadG{ss, reinterpret_cast<long long *>(c.subidx)}))) return rc;
    put_i64_kernel<<<1, 1, 0, c.st>>>(ss + nsub, c.K);
    if (nsub > 0)
        subject_n_kernel<<<grid_for(nsub), kTB, 0, c.st>>>(nsub, ss, c.y, reinterpret_cast<long long *>(c.sub_n),
                                                           c.flags);
    ScanBuf kb;
    long long Nk = 0;
    const long long *sn = reinterpret_cast<const long long *>(c.sub_n);
    if ((rc = scan_count(c, kb, KeepF{sn}, nsub, Nk))) return rc;
    if ((rc = scan_apply(c, kb, KeepF{sn}, KeepG{reinterpret_cast<long long *>(c.sub_new)}))) return rc;
    c.Nk = Nk;
    long long Kk = 0;
    if ((rc = scan_count(c, c.rows_sb, RowsF{sn, ss}, nsub, Kk))) return rc;
    c.Kk = Kk;
    return read_flags(c);
}

int subjects_fill(Ctx &c, int64_t *pat_ptr, int32_t *nev, int64_t *kept_from, double *Lk) {
    const long long *sn = reinterpret_cast<const long long *>(c.sub_n);
    const long long *ss = reinterpret_cast<const long long *>(c.sub_start);
    long long *pp = reinterpret_cast<long long *>(pat_ptr);
    int rc;
    if ((rc = scan_apply(c, c.rows_sb, RowsF{sn, ss},
                         RowsG{sn, reinterpret_cast<const long long *>(c.sub_new), pp,
                               reinterpret_cast<long long *>(kept_from), nev})))
        return rc;
    put_i64_kernel<<<1, 1, 0, c.st>>>(pp + c.Nk, c.Kk);
    const bool map_rows = c.Kk < c.K;
    if (map_rows && !(c.newrow = c.scr->get_n<int32_t>(static_cast<size_t>(c.K))))
        return static_cast<int>(cudaErrorMemoryAllocation);
    c.ksub = c.scr->get_n<int32_t>(static_cast<size_t>(c.Kk));
    c.ky = c.scr->get_n<int32_t>(static_cast<size_t>(c.Kk));
    if (!c.ksub || !c.ky) return static_cast<int>(cudaErrorMemoryAllocation);
    if (c.K > 0)
        kept_rows_kernel<<<grid_for(c.K), kTB, 0, c.st>>>(
            c.K, reinterpret_cast<const long long *>(c.subidx), ss, reinterpret_cast<const long long *>(c.sub_new), pp,
            c.y, c.L, map_rows ? c.newrow : nullptr, c.ksub, c.ky, Lk);
    return static_cast<int>(cudaGetLastError());
}

static void fill_down(std::vector<int64_t> &v, int64_t last) {
    // entries left at -1 belong to empty columns: they take the next entry's value
    const size_t n = v.size();
    v[n - 1] = last;
    for (size_t j = n - 1; j-- > 0;)
        if (v[j] < 0) v[j] = v[j + 1];
}

int columns(Ctx &c, std::vector<int64_t> &cptr_h, std::vector<int64_t> &ytx_h) {
    const int J = c.J;
    const size_t J1 = static_cast<size_t>(J) + 1;
    cptr_h.assign(J1, 0);
    c.cptr = c.scr->get_n<int64_t>(J1);
    if (!c.cptr) return static_cast<int>(cudaErrorMemoryAllocation);
    cudaError_t e;
    if (c.Kk == c.K) {                        // every row kept: the input columns as they are
        c.nnz = c.nnz_in;
        c.crow = const_cast<int32_t *>(c.ri);
        e = cudaMemcpyAsync(c.cptr, c.col_ptr, 8 * J1, cudaMemcpyDeviceToDevice, c.st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(cptr_h.data(), c.col_ptr, 8 * J1, cudaMemcpyDeviceToHost, c.st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
        if (e != cudaSuccess) return static_cast<int>(e);
    } else {
        std::vector<int64_t> first(J1, -1);
        e = cudaMemcpyAsync(c.cptr, first.data(), 8 * J1, cudaMemcpyHostToDevice, c.st);
        if (e != cudaSuccess) return static_cast<int>(e);
        ScanBuf sb;
        long long nnz = 0;
        const long long *cp = reinterpret_cast<const long long *>(c.col_ptr);
        KeepNzF f{c.ri, c.newrow};
        int rc = scan_count(c, sb, f, c.nnz_in, nnz);
        if (rc) return rc;
        c.nnz = nnz;
        c.crow = c.scr->get_n<int32_t>(static_cast<size_t>(nnz));
        if (!c.crow) return static_cast<int>(cudaErrorMemoryAllocation);
        if ((rc = scan_apply(c, sb, f, KeepNzG{c.ri, c.newrow, cp, J, c.crow, reinterpret_cast<long long *>(c.cptr)})))
            return rc;
        e = cudaMemcpyAsync(cptr_h.data(), c.cptr, 8 * J1, cudaMemcpyDeviceToHost, c.st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
        if (e != cudaSuccess) return static_cast<int>(e);
        fill_down(cptr_h, nnz);
        e = cudaMemcpyAsync(c.cptr, cptr_h.data(), 8 * J1, cudaMemcpyHostToDevice, c.st);
        if (e != cudaSuccess) return static_cast<int>(e);
    }
    const long long *cp = reinterpret_cast<const long long *>(c.cptr);
    uint8_t *unsorted = c.scr->get_n<uint8_t>(static_cast<size_t>(std::max(J, 1)));
    if (!unsorted) return static_cast<int>(cudaErrorMemoryAllocation);
    e = cudaMemsetAsync(unsorted, 0, static_cast<size_t>(std::max(J, 1)), c.st);
    if (e != cudaSuccess) return static_cast<int>(e);
    if (c.nnz > 0) column_check_kernel<<<grid_for(c.nnz), kTB, 0, c.st>>>(c.nnz, J, cp, c.crow, unsorted, c.flags);
    int rc = read_flags(c);
    if (rc) return rc;
    if (c.flags_h[kFUnsorted]) {
        // some column's rows are not ascending: those columns are sorted on the host, once
        std::vector<uint8_t> uns(static_cast<size_t>(std::max(J, 1)));
        std::vector<int32_t> rows(static_cast<size_t>(c.nnz));
        e = cudaMemcpyAsync(uns.data(), unsorted, uns.size(), cudaMemcpyDeviceToHost, c.st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(rows.data(), c.crow, 4 * rows.size(), cudaMemcpyDeviceToHost, c.st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
        if (e != cudaSuccess) return static_cast<int>(e);
        for (int j = 0; j < J; ++j)
            if (uns[j]) std::sort(rows.begin() + cptr_h[j], rows.begin() + cptr_h[j + 1]);
        e = cudaMemcpyAsync(c.crow, rows.data(), 4 * rows.size(), cudaMemcpyHostToDevice, c.st);
        if (e == cudaSuccess) e = cudaMemsetAsync(unsorted, 0, static_cast<size_t>(std::max(J, 1)), c.st);
        if (e != cudaSuccess) return static_cast<int>(e);
        column_check_kernel<<<grid_for(c.nnz), kTB, 0, c.st>>>(c.nnz, J, cp, c.crow, unsorted, c.flags);
        if ((rc = read_flags(c))) return rc;
    }
    if (c.flags_h[kFDup] != kNone) return 0;   // the caller reports the duplicate
    c.csub = c.scr->get_n<int32_t>(static_cast<size_t>(c.nnz));
    c.cy = c.scr->get_n<int32_t>(static_cast<size_t>(c.nnz));
    unsigned long long *ytx = c.scr->get_n<unsigned long long>(static_cast<size_t>(std::max(J, 1)));
    if (!c.csub || !c.cy || !ytx) return static_cast<int>(cudaErrorMemoryAllocation);
    e = cudaMemsetAsync(ytx, 0, 8 * static_cast<size_t>(std::max(J, 1)), c.st);
    if (e != cudaSuccess) return static_cast<int>(e);
    if (c.nnz > 0)
        column_lookup_kernel<<<grid_for(c.nnz), kTB, 0, c.st>>>(c.nnz, J, cp, c.crow, c.ksub, c.ky, c.csub, c.cy, ytx);
    ytx_h.assign(static_cast<size_t>(J), 0);
    if (J > 0) e = cudaMemcpyAsync(ytx_h.data(), ytx, 8 * static_cast<size_t>(J), cudaMemcpyDeviceToHost, c.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
    return static_cast<int>(e);
}

int segments(Ctx &c, std::vector<int64_t> &cseg_ptr_h) {
    const int J = c.J;
    const size_t J1 = static_cast<size_t>(J) + 1;
    const long long *cp = reinterpret_cast<const long long *>(c.cptr);
    ScanBuf sb;
    long long nseg = 0;
    SegHeadF f{cp, c.csub, J};
    int rc = scan_count(c, sb, f, c.nnz, nseg);
    if (rc) return rc;
    c.nseg = nseg;
    c.cs_start = c.scr->get_n<int64_t>(static_cast<size_t>(nseg) + 1);
    c.cs_sub = c.scr->get_n<int32_t>(static_cast<size_t>(nseg));
    c.cs_len = c.scr->get_n<int32_t>(static_cast<size_t>(nseg));
    c.cs_y = c.scr->get_n<int32_t>(static_cast<size_t>(nseg));
    c.cseg_ptr = c.scr->get_n<int64_t>(J1);
    if (!c.cs_start || !c.cs_sub || !c.cs_len || !c.cs_y || !c.cseg_ptr)
        return static_cast<int>(cudaErrorMemoryAllocation);
    std::vector<int64_t> first(J1, -1);
    cudaError_t e = cudaMemcpyAsync(c.cseg_ptr, first.data(), 8 * J1, cudaMemcpyHostToDevice, c.st);
    if (e != cudaSuccess) return static_cast<int>(e);
    long long *cs = reinterpret_cast<long long *>(c.cs_start);
    if ((rc = scan_apply(c, sb, f, SegHeadG{cp, c.csub, J, cs, reinterpret_cast<long long *>(c.cseg_ptr), c.cs_sub})))
        return rc;
    put_i64_kernel<<<1, 1, 0, c.st>>>(cs + nseg, c.nnz);
    if (nseg > 0)
        segment_values_kernel<<<grid_for(nseg), kTB, 0, c.st>>>(nseg, cs, c.cy, c.cs_len, c.cs_y, c.flags);
    cseg_ptr_h.assign(J1, 0);
    e = cudaMemcpyAsync(cseg_ptr_h.data(), c.cseg_ptr, 8 * J1, cudaMemcpyDeviceToHost, c.st);
    if (e != cudaSuccess) return static_cast<int>(e);
    if ((rc = read_flags(c))) return rc;
    fill_down(cseg_ptr_h, nseg);
    c.lmax = static_cast<int32_t>(c.flags_h[kFLmax]);
    e = cudaMemcpyAsync(c.cseg_ptr, cseg_ptr_h.data(), 8 * J1, cudaMemcpyHostToDevice, c.st);
    return static_cast<int>(e);
}

int pairs_count(Ctx &c, ScanBuf &sb, int64_t &npairs) {
    long long n = 0;
    int rc = scan_count(c, sb, PairF{c.cs_y}, c.nseg, n);
    npairs = n;
    return rc;
}

int pairs_fill(Ctx &c, ScanBuf &sb, int64_t npairs, int32_t *ysub, int32_t *ycnt, std::vector<int64_t> &ycol_ptr_h) {
    const size_t J1 = static_cast<size_t>(c.J) + 1;
    long long *first = c.scr->get_n<long long>(J1);
    if (!first) return static_cast<int>(cudaErrorMemoryAllocation);
    ycol_ptr_h.assign(J1, -1);
    cudaError_t e = cudaMemcpyAsync(first, ycol_ptr_h.data(), 8 * J1, cudaMemcpyHostToDevice, c.st);
    if (e != cudaSuccess) return static_cast<int>(e);
    int rc = scan_apply(c, sb, PairF{c.cs_y},
                        PairG{c.cs_y, c.cs_sub, reinterpret_cast<const long long *>(c.cseg_ptr), c.J, ysub, ycnt, first});
    if (rc) return rc;
    e = cudaMemcpyAsync(ycol_ptr_h.data(), first, 8 * J1, cudaMemcpyDeviceToHost, c.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
    if (e != cudaSuccess) return static_cast<int>(e);
    fill_down(ycol_ptr_h, npairs);
    return 0;
}

int shards(Ctx &c, const int64_t *pat_ptr, int32_t Sp, int64_t *shard_pat, int64_t *shard_row) {
    shards_kernel<<<(Sp + 1 + 127) / 128, 128, 0, c.st>>>(reinterpret_cast<const long long *>(pat_ptr), c.Nk, c.Kk, Sp,
                                      reinterpret_cast<long long *>(shard_pat), reinterpret_cast<long long *>(shard_row));
    return static_cast<int>(cudaGetLastError());
}

int slices_count(Ctx &c, SliceSet &ss, std::vector<int64_t> *nnz_h, std::vector<int64_t> *nseg_h) {
    const long long nsl = static_cast<long long>(ss.Sp) * (c.J + 1);
    ss.sl_a = c.scr->get_n<int64_t>(static_cast<size_t>(nsl));
    ss.sl_nnz = c.scr->get_n<int64_t>(static_cast<size_t>(nsl));
    ss.sl_nseg = c.scr->get_n<int64_t>(static_cast<size_t>(nsl));
    if (!ss.sl_a || !ss.sl_nnz || !ss.sl_nseg) return static_cast<int>(cudaErrorMemoryAllocation);
    flags_init_kernel<<<1, 32, 0, c.st>>>(c.flags);   // resets the maxima (and the other words)
    slice_count_kernel<<<grid_for(nsl), kTB, 0, c.st>>>(
        ss.Sp, c.J, reinterpret_cast<const long long *>(ss.shard_pat), ss.mask,
        reinterpret_cast<const long long *>(c.cseg_ptr), c.cs_sub, reinterpret_cast<const long long *>(c.cs_start),
        reinterpret_cast<long long *>(ss.sl_a), reinterpret_cast<long long *>(ss.sl_nnz),
        reinterpret_cast<long long *>(ss.sl_nseg), c.flags);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return static_cast<int>(e);
    if (nnz_h) {
        nnz_h->assign(static_cast<size_t>(nsl), 0);
        e = cudaMemcpyAsync(nnz_h->data(), ss.sl_nnz, 8 * static_cast<size_t>(nsl), cudaMemcpyDeviceToHost, c.st);
        if (e != cudaSuccess) return static_cast<int>(e);
    }
    if (nseg_h) {
        nseg_h->assign(static_cast<size_t>(nsl), 0);
        e = cudaMemcpyAsync(nseg_h->data(), ss.sl_nseg, 8 * static_cast<size_t>(nsl), cudaMemcpyDeviceToHost, c.st);
        if (e != cudaSuccess) return static_cast<int>(e);
    }
    int rc = read_flags(c);
    if (rc) return rc;
    ss.max_seg = static_cast<int64_t>(c.flags_h[kFMaxSeg]);
    ss.max_rows = static_cast<int64_t>(c.flags_h[kFMaxRows]);
    long long t = 0;
    if ((rc = scan_count(c, ss.sc_row, ArrF{reinterpret_cast<const long long *>(ss.sl_nnz)}, nsl, t))) return rc;
    ss.tr = t;
    if ((rc = scan_count(c, ss.sc_seg, ArrF{reinterpret_cast<const long long *>(ss.sl_nseg)}, nsl, t))) return rc;
    ss.ts = t;
    if ((rc = scan_count(c, ss.sc_grp, GrpF{reinterpret_cast<const long long *>(ss.sl_nseg)}, nsl, t))) return rc;
    ss.tg = t;
    return 0;
}

int slices_fill(Ctx &c, SliceSet &ss, int64_t *slice_row, int64_t *slice_seg, int64_t *slice_grp, int32_t *rows,
                int2 *segs, int64_t *grp_base) {
    const long long nsl = static_cast<long long>(ss.Sp) * (c.J + 1);
    long long *sr = reinterpret_cast<long long *>(slice_row), *sg = reinterpret_cast<long long *>(slice_seg),
              *sgr = reinterpret_cast<long long *>(slice_grp);
    int rc;
    if ((rc = scan_apply(c, ss.sc_row, ArrF{reinterpret_cast<const long long *>(ss.sl_nnz)}, PutG{sr}))) return rc;
    if ((rc = scan_apply(c, ss.sc_seg, ArrF{reinterpret_cast<const long long *>(ss.sl_nseg)}, PutG{sg}))) return rc;
    if ((rc = scan_apply(c, ss.sc_grp, GrpF{reinterpret_cast<const long long *>(ss.sl_nseg)}, PutG{sgr}))) return rc;
    if (ss.ts == 0) return 0;
    long long *sorted = c.scr->get_n<long long>(static_cast<size_t>(ss.ts));
    long long *grows = c.scr->get_n<long long>(static_cast<size_t>(ss.tg));
    if (!sorted || !grows) return static_cast<int>(cudaErrorMemoryAllocation);
    // per-warp length bins: shared memory, or (very long segments) a global array per warp
    const bool use_smem = c.lmax < kBins;
    int sort_blocks = grid_for(nsl, kWarpsPB);
    int *gbins = nullptr;
    long long gstride = 0;
    if (!use_smem) {
        gstride = static_cast<long long>(c.lmax) + 1;
        const long long max_warps = std::max<long long>(kWarpsPB, (256ll << 20) / (4 * gstride));
        sort_blocks = static_cast<int>(std::max<long long>(1, std::min<long long>(sort_blocks, max_warps / kWarpsPB)));
        gbins = c.scr->get_n<int>(static_cast<size_t>(sort_blocks) * kWarpsPB * static_cast<size_t>(gstride));
        if (!gbins) return static_cast<int>(cudaErrorMemoryAllocation);
    }
    slice_sort_kernel<<<sort_blocks, kTB, 0, c.st>>>(nsl, c.J, reinterpret_cast<const long long *>(ss.sl_a), sg,
                                                     c.cs_len, c.cs_sub, segs, sorted, gbins, gstride, use_smem);
    const int gblocks = grid_for(ss.tg, kWarpsPB);
    group_rows_kernel<<<gblocks, kTB, 0, c.st>>>(ss.tg, nsl, sgr, sg, segs, grows);
    ScanBuf gb;
    long long t = 0;
    if ((rc = scan_count(c, gb, ArrF{grows}, ss.tg, t))) return rc;
    if ((rc = scan_apply(c, gb, ArrF{grows}, PutG{reinterpret_cast<long long *>(grp_base)}))) return rc;
    jds_fill_kernel<<<gblocks, kTB, 0, c.st>>>(ss.tg, nsl, sgr, sg, segs, sorted,
                                               reinterpret_cast<const long long *>(c.cs_start),
                                               reinterpret_cast<const long long *>(grp_base), c.crow, rows);
    return static_cast<int>(cudaGetLastError());
}

int last_prev_columns(Ctx &c, const int64_t *pat_ptr, const int64_t *row_ptr, const int32_t *row_col,
                      const std::vector<int32_t> &cols, std::vector<int32_t> &lp) {
    const int n = static_cast<int>(cols.size());
    lp.assign(cols.size(), -1);
    if (n == 0) return 0;
    int *dcols = c.scr->get_n<int>(cols.size());
    int *dlp = c.scr->get_n<int>(cols.size());
    if (!dcols || !dlp) return static_cast<int>(cudaErrorMemoryAllocation);
    cudaError_t e = cudaMemcpyAsync(dcols, cols.data(), 4 * cols.size(), cudaMemcpyHostToDevice, c.st);
    if (e != cudaSuccess) return static_cast<int>(e);
    last_prev_kernel<<<std::min(n, 152 * 8), kTB, 0, c.st>>>(
        dcols, n, reinterpret_cast<const long long *>(c.cptr), c.csub, reinterpret_cast<const long long *>(pat_ptr),
        reinterpret_cast<const long long *>(row_ptr), row_col, dlp);
    e = cudaMemcpyAsync(lp.data(), dlp, 4 * cols.size(), cudaMemcpyDeviceToHost, c.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
    return static_cast<int>(e);
}

int narrow_fill(Ctx &c, const int64_t *pat_ptr, const int64_t *row_ptr, const int32_t *row_col,
                const std::vector<NarrowCol> &cols, int4 *nar_seg, int32_t *nar_row, int32_t after_wide) {
    const int n = static_cast<int>(cols.size());
    if (n == 0) return 0;
    std::vector<NarrowColDev> h(cols.size());
    for (size_t i = 0; i < cols.size(); ++i)
        h[i] = NarrowColDev{cols[i].j, cols[i].run_wide, cols[i].prev0, cols[i].prevm, cols[i].nar_first,
                            cols[i].row_first};
    NarrowColDev *d = c.scr->get_n<NarrowColDev>(h.size());
    if (!d) return static_cast<int>(cudaErrorMemoryAllocation);
    cudaError_t e = cudaMemcpyAsync(d, h.data(), sizeof(NarrowColDev) * h.size(), cudaMemcpyHostToDevice, c.st);
    if (e != cudaSuccess) return static_cast<int>(e);
    narrow_fill_kernel<<<std::min(n, 152 * 8), kTB, 0, c.st>>>(
        d, n, reinterpret_cast<const long long *>(c.cptr), reinterpret_cast<const long long *>(c.cseg_ptr),
        reinterpret_cast<const long long *>(c.cs_start), c.cs_sub, c.cs_len, c.crow,
        reinterpret_cast<const long long *>(pat_ptr), reinterpret_cast<const long long *>(row_ptr), row_col, nar_seg,
        nar_row, after_wide);
    return static_cast<int>(cudaGetLastError());
}

}  // namespace lay
}  // namespace sccs
