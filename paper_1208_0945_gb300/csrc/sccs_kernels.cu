// sccs_kernels.cu -- sm_103a kernels for the BSCCS cyclic-coordinate-descent MAP fit.
//
// One persistent cooperative launch runs a whole fit (Algorithm 1).  CTA s owns subject
// shard s: the eras (rows) and subjects in it, their L x exp(Xb) (E) and M[L x exp(Xb)] (D).
// Per coordinate j every CTA
//   A  gathers E at the nonzeros of its slice of X_j, sums them per subject (the numerator
//      M[L x exp(Xb) x X_j] of Eq. 8, restricted to the touched subjects), forms
//      W_i = num_i / D_i and the partial sums  sum n_i W_i  and  sum n_i W_i (1 - W_i)
//      (the fused transformation and reduction of Section 2.4, with W never stored);
//   -  joins one grid all-reduce of the two partials, then one lane computes g_j, h_j
//      (Eqs. 7, 9) and the step db_j (Eq. 4 with the prior of Eq. 3 and a Genkin trust
//      region) and broadcasts db_j, e^{db_j} and e^{db_j} - 1;
//   C  if db_j != 0, updates its own rows and subjects (Section 2.3 steps 1-3):
//      E_k <- E_k e^{db}  (= l_k exp(Xb_k + db): one exp per coordinate instead of one per
//      nonzero), and D_i <- D_i + (e^{db} - 1) num_i (= D_i + sum_k (E_k,new - E_k,old)).
// No CTA ever touches another shard's rows, so phase C needs no grid barrier: the only
// cross-CTA traffic is 16 bytes per CTA per coordinate.  At the end of a cycle each CTA
// recomputes D from E on its subjects and the log-posterior is all-reduced.
//
// GB300 specifics:
//   * The static part of a column's slice (segments, rows, group offsets) is staged into
//     shared memory by bulk asynchronous copies (cp.async.bulk + mbarrier) one column ahead,
//     so only the gathers of the state E and D remain on the critical path.
//   * An FP64 instruction holds its SM sub-partition's FP64 pipe about as long with one active
//     lane as with 32.  The coordinate path's sums (lane -> warp -> CTA -> cluster or grid) are
//     therefore lane trees in FP64, one instruction per level, in orders fixed by the launch
//     shape (lane butterflies, warps in warp order, CTAs by cluster rank or shard), never by
//     arrival: all CTAs obtain bit-identical totals and every run is repeatable bit for bit.
//     Warps that took no segment skip their tree.  Exact 192-bit fixed point (integer
//     instructions) remains for the cycle-end log-posterior, the narrow columns and the FP32
//     mode's per-thread sums.  FP64 is kept for the per-subject arithmetic and the scalar step,
//     which one lane computes once per coordinate.
//
// Every wait is bounded by a deadline on %globaltimer; a CTA that gives up raises the abort
// flag, waits (bounded) for its own bulk copies in flight and returns; the others see the
// flag and return too.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "sccs.h"
#include "sccs_internal.h"

namespace sccs {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kBatch = 8;        // diagonals gathered per batch
constexpr int kMaxWarps = 32;
constexpr int kFrac = 128;       // fraction bits of the fixed-point sums (value = V * 2^-128)
// E_k <- E_k e^{db} rounds once per update; every so many cycles E is rebuilt from beta instead
// (FP64: at most 1.5 ulp per update, so 64 cycles of a row in c columns drift <= 96 c ulp; FP32
// rounds 2^29 times coarser, so it is rebuilt 4 times as often)
constexpr int kRebuildCycles64 = 64;
constexpr int kRebuildCycles32 = 16;

// status values written to FitOut
constexpr int kStOk = 0;
constexpr int kStNotConverged = 1;
constexpr int kStTimeout = -6;
constexpr int kStNumeric = -7;

// ------------------------------------------------------------------ timers, memory order

__device__ __forceinline__ long long now_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void ld_relaxed_v2(const unsigned long long *p, unsigned long long &a,
                                              unsigned long long &b) {
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}

__device__ __forceinline__ void st_relaxed_v2(unsigned long long *p, unsigned long long a, unsigned long long b) {
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}

__device__ __forceinline__ int ld_relaxed_i32(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Barrier 1 among warps 1..n-1 (warp 0 is busy with the all-reduce).
// 4-byte asynchronous global -> shared copies (no registers held while in flight).
__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gmem_src) {
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
#if SCCS_L2HINT >= 1
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 4, %2;" ::"r"(sa), "l"(gmem_src), "l"(pol)
                 : "memory");
#else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem_src) : "memory");
#endif
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void named_barrier_all_but_warp0() {
    asm volatile("bar.sync 1, %0;" ::"r"(static_cast<int>(blockDim.x) - 32) : "memory");
}

__device__ __forceinline__ void prefetch_l1(const void *p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Into L2 only: L2 is where all SMs' writes meet, so an early copy there cannot go stale.
__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// ------------------------------------------------------------------ bulk copies, mbarriers

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

#ifndef SCCS_L2HINT
#define SCCS_L2HINT 0
#endif
#ifndef SCCS_REGATHER_E
#define SCCS_REGATHER_E 0
#endif
// L2 eviction priorities: the static structure is read once per cycle and streamed past the
// state (E, D), which is read and written at every step
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint64_t l2_evict_last() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
template <class T>
__device__ __forceinline__ T ld_static(const T *p) {
#if SCCS_L2HINT >= 1
    return __ldcs(p);
#else
    return *p;
#endif
}
__device__ __forceinline__ double ld_state(const double *p) {
#if SCCS_L2HINT >= 2
    double v;
    asm volatile("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(l2_evict_last()));
    return v;
#else
    return *p;
#endif
}
__device__ __forceinline__ void st_state(double *p, double v) {
#if SCCS_L2HINT >= 2
    asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(l2_evict_last()) : "memory");
#else
    *p = v;
#endif
}

// Global -> shared bulk copy; dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
#if SCCS_L2HINT >= 1
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
        "%4;" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(l2_evict_first())
        : "memory");
#else
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
#endif
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of a bulk-copy barrier.
__device__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long deadline = now_ns() + timeout_ns;
    for (int it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 31) == 31 && now_ns() > deadline) return false;
    }
}

// ------------------------------------------------------------------ thread-block clusters

// The shared::cluster address of `local` (this CTA's shared memory) in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t cluster_addr(const void *local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_addr(local)), "r"(rank));
    return r;
}

// 16 bytes into another CTA's shared memory, counted (complete_tx) on an mbarrier of that CTA:
// the receiver sees the bytes once that mbarrier's phase completes.
__device__ __forceinline__ void st_async_f64x2(uint32_t addr, double a, double b, uint32_t remote_bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];" ::"r"(addr),
                 "d"(a), "d"(b), "r"(remote_bar)
                 : "memory");
}

// Every thread of every CTA of the cluster (hardware barrier; used only where all of them arrive
// unconditionally: after the mbarrier initialisation and before the kernel exits).
__device__ __forceinline__ void cluster_barrier_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// ------------------------------------------------------------------ exact fixed-point sums

// A non-negative value V * 2^-128 held in three 64-bit limbs (w0 least significant).
struct Fx {
    unsigned long long w0, w1, w2;
};

__device__ __forceinline__ Fx fx_zero() { return Fx{0ull, 0ull, 0ull}; }

__device__ __forceinline__ Fx fx_add(const Fx &a, const Fx &b) {
    Fx r;
    r.w0 = a.w0 + b.w0;
    const unsigned long long c0 = r.w0 < a.w0;
    const unsigned long long t1 = a.w1 + b.w1;
    const unsigned long long c1a = t1 < a.w1;
    r.w1 = t1 + c0;
    const unsigned long long c1b = r.w1 < t1;
    r.w2 = a.w2 + b.w2 + c1a + c1b;
    return r;
}

// Exact conversion of a finite non-negative double below 2^60; bits below 2^-128 are
// dropped.  Anything else (negative, NaN, inf, huge) sets `bad`.
__device__ __forceinline__ Fx fx_from_double(double v, bool &bad) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
    const int e = static_cast<int>((b >> 52) & 0x7ff);
    Fx r = fx_zero();
    if ((b >> 63) && b != 0x8000000000000000ull) {  // negative (minus zero is zero)
        bad = true;
        return r;
    }
    if (e == 0) return r;                        // zero or subnormal
    if (e >= 1023 + 60) {                        // >= 2^60, inf or NaN
        bad = true;
        return r;
    }
    const unsigned long long m = (b & 0xfffffffffffffull) | (1ull << 52);
    const int sh = e - 1075 + kFrac;             // v = m * 2^(e - 1075)
    if (sh < 0) {
        if (sh > -64) r.w0 = m >> (-sh);
        return r;
    }
    const int q = sh >> 6, rm = sh & 63;
    const unsigned long long lo = m << rm;
    const unsigned long long hi = rm ? (m >> (64 - rm)) : 0ull;
    if (q == 0) {
        r.w0 = lo;
        r.w1 = hi;
    } else if (q == 1) {
        r.w1 = lo;
        r.w2 = hi;
    } else {
        r.w2 = lo;
    }
    return r;
}

// Round-to-nearest-even conversion back to double.
__device__ __forceinline__ double fx_to_double(const Fx &v) {
    int p;
    if (v.w2) p = 128 + 63 - __clzll(static_cast<long long>(v.w2));
    else if (v.w1) p = 64 + 63 - __clzll(static_cast<long long>(v.w1));
    else if (v.w0) p = 63 - __clzll(static_cast<long long>(v.w0));
    else return 0.0;
    // W = bits [p-63, p] of V; sticky = any bit below p-63
    unsigned long long W;
    bool sticky = false;
    if (p < 63) {
        W = v.w0 << (63 - p);
    } else {
        const int s = p - 63;
        const int q = s >> 6, r = s & 63;
        const unsigned long long L0 = q == 0 ? v.w0 : (q == 1 ? v.w1 : v.w2);
        const unsigned long long L1 = q == 0 ? v.w1 : (q == 1 ? v.w2 : 0ull);
        W = r ? ((L0 >> r) | (L1 << (64 - r))) : L0;
        const unsigned long long below = r ? (L0 & ((1ull << r) - 1)) : 0ull;
        sticky = below != 0 || (q >= 1 && v.w0 != 0) || (q >= 2 && v.w1 != 0);
    }
    unsigned long long m = W >> 11;
    const unsigned long long rb = (W >> 10) & 1ull;
    sticky = sticky || (W & 0x3ffull) != 0;
    long long biased = static_cast<long long>(p) - kFrac + 1023;
    if (rb && (sticky || (m & 1ull))) {
        m += 1;
        if (m == (1ull << 53)) {
            m >>= 1;
            biased += 1;
        }
    }
    const unsigned long long bits = (static_cast<unsigned long long>(biased) << 52) | (m & 0xfffffffffffffull);
    return __longlong_as_double(static_cast<long long>(bits));
}

__device__ __forceinline__ Fx fx_shfl_down(const Fx &v, int o) {
    Fx r;
    r.w0 = __shfl_down_sync(kFull, v.w0, o);
    r.w1 = __shfl_down_sync(kFull, v.w1, o);
    r.w2 = __shfl_down_sync(kFull, v.w2, o);
    return r;
}

// Exact warp sum; the total is in lane 0.
__device__ __forceinline__ Fx fx_warp_sum(Fx v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fx_add(v, fx_shfl_down(v, o));
    return v;
}

// Warp sum by a fixed FP64 tree (xor butterfly): lane 0's order of additions is always the same,
// so its result is a deterministic function of the 32 inputs; only lane 0's result is used.
__device__ __forceinline__ double warp_tree_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// A warp's two partial sums (lane 0's result).  A warp whose lanes all hold +0 (it took no
// segment) skips the tree: each FP64 instruction holds the SM partition's FP64 pipe as long with
// one lane as with 32, and the idle warps of a small column would otherwise queue ten of them each
// in front of the warps with data.  The test is on bit patterns (integer instructions); the sum of
// +0s is +0 either way, so the result is the same.
// The tree also stops at the highest lane that holds data: with data in lanes 0..n-1 only (a
// small slice), log2 n levels give lane 0 the same sum as five (the other lanes add +0 exactly).
__device__ __forceinline__ void warp_tree_sum2(double &a, double &b, bool bad) {
    const bool some = __double_as_longlong(a) != 0 || __double_as_longlong(b) != 0 || bad;
    const unsigned m = __ballot_sync(kFull, some);
    if (m != 0u) {
        const int top = 31 - __clz(static_cast<int>(m));     // highest lane with data
        for (int o = top > 0 ? 1 << (31 - __clz(top)) : 0; o > 0; o >>= 1) {
            a += __shfl_xor_sync(kFull, a, o);
            b += __shfl_xor_sync(kFull, b, o);
        }
    }
}

// The same over lanes 0..15 only (4 levels; lane 0's result).  An FP64 instruction costs its SM
// partition the same issue time whatever the number of active lanes, so a tree across lanes (one
// instruction per level) is much cheaper than one lane adding the values in turn.
__device__ __forceinline__ double warp_tree_sum16(double v) {
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// ------------------------------------------------------------------ shared state

struct StageBuf {
    int2 segs[kSegCap + 2];          // 16,400 B
    int32_t rows[kRowCap + 8];       // 16,416 B
    long long grp[kGrpCap + 2];      //    528 B
};

struct ColDesc {
    long long seg0, row0, grp0;
    int nseg, nnz, ngrp, staged;
    int seg_off, row_off, grp_off, cl;   // cl: a slice of the cluster partition
    int gm;                              // columns of a cluster group (1 otherwise)
};

// A staged cluster group: column t's JDS groups, segments and rows within the staged slice.
struct GroupOffs {
    int goff[kNarrowGroupMax + 1], soff[kNarrowGroupMax + 1], roff[kNarrowGroupMax + 1];
};

struct SharedState {
    Fx wa[kMaxWarps];
    Fx wb[kMaxWarps];
    int wbad[kMaxWarps];
    double wda[kMaxWarps], wdb[kMaxWarps];   // per warp: its FP64 sums (the coordinate path)
    double db, r, em1;
    // a group of narrow (or cluster) columns: per column step results, and the group's flags
    double gdb[kNarrowGroupMax], gr[kNarrowGroupMax], gem1[kNarrowGroupMax], gnbj[kNarrowGroupMax],
        gtrust[kNarrowGroupMax];
    double gb[kNarrowGroupMax], gt[kNarrowGroupMax], gy[kNarrowGroupMax];   // a cluster group's b_j, T_j, Y'X_j
    int gnumeric, gwarn, gnonzero;
    double G, H;
    double lin, sq, ab;     // cycle sums of b_j Y'X_j, b_j^2, |b_j| (from the bookkeeping thread)
    long long nonzero;
    int ok;
    int stop;
    ColDesc desc[2];
    GroupOffs gofs[2];
    uint64_t bar[2];
    int run_status;         // a finished run_fit's status (thread 0 writes it)
    int drained;            // its staging copies all landed (thread blockDim - 32 writes it)
    unsigned long long run_seq;   // the all-reduce sequence number it ended at
    int nar_pre;            // CTA 0: the narrow run whose first group's static data is in nar_hi
    // cluster all-reduce: each CTA's pair of partials, written by every CTA of the cluster into
    // every CTA's slots, and the mbarriers that count their bytes (both by round parity)
    double2 cslot[2][kNarrowGroupMax][16];
    uint64_t cbar[2];
};

// One narrow group's gathered data (half of the narrow buffers).
struct NarrowBuf {
    double est[kRowCap / 2];             // E per row
    double2 stash[kSegCap / 2];          // (numerator, D) per segment
    int4 info[kSegCap / 2];              // {subject, rows | mark << 16, first row, n_i} per segment
    int rows[kRowCap / 2];               // index into E per row
    int m;                               // columns in the group
    int col_off[kNarrowGroupMax + 1];    // each column's first segment
};

// A wide column's gathered state between its phases A and C (for a slice too big to stage, the
// row-index ring of phase_a_global: 2 x 32 x kBatch ints per warp).
struct WideBuf {
    double est[kRowCap];             // E gathered in phase A, per row position
    double2 seg_stash[kSegCap];      // (num, D) per segment
};
static_assert(kMaxWarps * 2 * 32 * kBatch * sizeof(int) <= sizeof(WideBuf), "row ring exceeds the wide buffer");

// Wide columns and narrow runs never hold gathered state at the same time (CTA 0 finishes a
// wide column's phase C before a narrow run starts, and the run before the next phase A), so
// one narrow buffer shares space with the wide one.  The other (nar_hi) takes a run's first
// group, whose static data is gathered while the wide column before the run is still live.
struct SmemLayout {
    StageBuf stage[2];
    union {
        WideBuf wide;
        NarrowBuf nar_lo;
    };
    NarrowBuf nar_hi;        // last: launches without narrow columns leave it out
    __device__ NarrowBuf &nar(int half) { return half ? nar_hi : nar_lo; }
};
static_assert(sizeof(SmemLayout) - sizeof(NarrowBuf) >= offsetof(SmemLayout, nar_hi),
              "the second narrow buffer is the layout's last member");

// ------------------------------------------------------------------ grid all-reduce

// Grid all-reduce of two non-negative partials, run by one full warp of every CTA.
// Slot buffer (seq & 1) holds this round; the sign bit of each value equals the round's
// phase ((seq >> 1) & 1) ^ 1, which differs from what the buffer held two rounds earlier,
// so a reader can tell a fresh value from a stale one without a separate flag.  A CTA can
// not run two rounds ahead of a reader, because the round after next needs the reader's
// own contribution.  The totals are FP64 sums in one fixed order over the slots (each lane its
// slots in ascending order, then a fixed tree over the lanes, whose lane-0 result every CTA
// takes), so every CTA holds the same bits, whatever the order the partials arrived in.  With `sync` the round is also a release/acquire: each CTA's writes
// before its contribution (ordered by a CTA barrier before the call) are visible to every
// CTA after the call (and, after a CTA barrier, to all its threads).
__device__ bool grid_allreduce2(const DevLayout &d, int me, unsigned long long seq, double a, double b, double &A,
                                double &B, long long timeout_ns, bool sync = false) {
    const int lane = threadIdx.x & 31;
    const unsigned long long phase = ((seq >> 1) & 1ull) ^ 1ull;
    unsigned long long *buf = d.slots + (seq & 1ull) * 2ull * static_cast<unsigned long long>(d.S);
    if (lane == 0) {
        const unsigned long long ea = (static_cast<unsigned long long>(__double_as_longlong(a)) &
                                       0x7fffffffffffffffull) | (phase << 63);
        const unsigned long long eb = (static_cast<unsigned long long>(__double_as_longlong(b)) &
                                       0x7fffffffffffffffull) | (phase << 63);
        if (sync) __threadfence();                    // release: the CTA's writes before the slot
        st_relaxed_v2(buf + 2 * me, ea, eb);
    }
    const long long deadline = now_ns() + timeout_ns;
    double sa = 0.0, sb = 0.0;
    for (int it = 0;; ++it) {
        bool ready = true;
        unsigned long long va[5], vb[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const int s = lane + 32 * q;
            va[q] = vb[q] = 0ull;
            if (s < d.S) ld_relaxed_v2(buf + 2 * s, va[q], vb[q]);
        }
        for (int s = lane + 160; s < d.S; s += 32) {   // more than 160 shards
            unsigned long long x, y;
            ld_relaxed_v2(buf + 2 * s, x, y);
            ready &= ((x >> 63) == phase) && ((y >> 63) == phase);
        }
#pragma unroll
        for (int q = 0; q < 5; ++q)
            if (lane + 32 * q < d.S) ready &= ((va[q] >> 63) == phase) && ((vb[q] >> 63) == phase);
        if (__all_sync(kFull, ready)) {
            // each lane adds its slots in ascending order, then a fixed tree over the lanes: lane
            // 0's order of additions is the same in every CTA (NaN, a bad partial, carries through)
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                if (lane + 32 * q < d.S) {
                    sa += __longlong_as_double(static_cast<long long>(va[q] & 0x7fffffffffffffffull));
                    sb += __longlong_as_double(static_cast<long long>(vb[q] & 0x7fffffffffffffffull));
                }
            }
            for (int s = lane + 160; s < d.S; s += 32) {
                unsigned long long x, y;
                ld_relaxed_v2(buf + 2 * s, x, y);
                sa += __longlong_as_double(static_cast<long long>(x & 0x7fffffffffffffffull));
                sb += __longlong_as_double(static_cast<long long>(y & 0x7fffffffffffffffull));
            }
            break;
        }
        int give_up = 0;
        if (lane == 0 && (it & 15) == 15)
            give_up = (ld_relaxed_i32(d.abort_flag) != 0) || (now_ns() > deadline);
        if (__shfl_sync(kFull, give_up, 0)) {
            if (lane == 0) atomicExch(d.abort_flag, 1);
            return false;
        }
    }
    if (sync) __threadfence();                        // acquire: after reading every slot
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sa += __shfl_xor_sync(kFull, sa, o);
        sb += __shfl_xor_sync(kFull, sb, o);
    }
    A = __shfl_sync(kFull, sa, 0);
    B = __shfl_sync(kFull, sb, 0);
    return true;
}

// Grid all-reduce of a launch in thread-block clusters of C CTAs (warp 0 of every CTA; S = k C).
// Two levels.  The C CTAs of a cluster first exchange their pairs through distributed shared
// memory: every CTA sends its pair to slot [0][rank] of every CTA of its cluster by asynchronous
// stores counted on that CTA's mbarrier of cluster round `round` (the cluster groups' protocol),
// and adds the C pairs in rank order by a lane tree, so each holds its cluster's total.  Then every
// CTA writes that total into its own global slot (phase-tagged as in grid_allreduce2, so every
// slot of the buffer carries the round's phase and the flat all-reduce may use the same slots
// next), and reads the k cluster totals from the slots of the clusters' first CTAs (one slot per
// lane, k <= 32), added by a lane tree.  Every order is fixed, so all CTAs hold the same bits.
// A CTA can not run two rounds ahead: the round after next needs every cluster's total of the
// next round, which needs every CTA's pair of it, sent only after it read this round.
__device__ bool cluster_grid_allreduce2(const DevLayout &d, SharedState &sh, int me, int rank, unsigned round,
                                        unsigned long long seq, double a, double b, double &A, double &B,
                                        long long timeout_ns) {
    const int lane = threadIdx.x & 31;
    const int C = d.C;
    const int ncl = d.S / C;
    // level 1: the cluster
    const int cbuf = static_cast<int>(round & 1u);
    const uint32_t parity = (round >> 1) & 1u;
    if (lane == 0) mbar_arrive_expect_tx(&sh.cbar[cbuf], static_cast<uint32_t>(16 * C));
    if (lane < C) st_async_f64x2(cluster_addr(&sh.cslot[cbuf][0][rank], lane), a, b, cluster_addr(&sh.cbar[cbuf], lane));
    int ok = 1;
    if (!mbar_try_wait(&sh.cbar[cbuf], parity)) {
        const long long deadline = now_ns() + timeout_ns;
        for (int it = 0;; ++it) {
            if (mbar_try_wait(&sh.cbar[cbuf], parity)) break;
            if ((it & 31) == 31 && (ld_relaxed_i32(d.abort_flag) != 0 || now_ns() > deadline)) {
                ok = 0;
                break;
            }
        }
    }
    if (!__all_sync(kFull, ok)) {
        if (lane == 0) atomicExch(d.abort_flag, 1);
        return false;
    }
    double ca = 0.0, cb = 0.0;
    if (lane < C) {
        const double2 v = sh.cslot[cbuf][0][lane];
        ca = v.x;
        cb = v.y;
    }
    ca = __shfl_sync(kFull, warp_tree_sum16(ca), 0);
    cb = __shfl_sync(kFull, warp_tree_sum16(cb), 0);
    // level 2: the clusters, through global memory
    const unsigned long long phase = ((seq >> 1) & 1ull) ^ 1ull;
    unsigned long long *buf = d.slots + (seq & 1ull) * 2ull * static_cast<unsigned long long>(d.S);
    if (lane == 0) {
        const unsigned long long ea = (static_cast<unsigned long long>(__double_as_longlong(ca)) &
                                       0x7fffffffffffffffull) | (phase << 63);
        const unsigned long long eb = (static_cast<unsigned long long>(__double_as_longlong(cb)) &
                                       0x7fffffffffffffffull) | (phase << 63);
        st_relaxed_v2(buf + 2 * me, ea, eb);
    }
    const long long deadline = now_ns() + timeout_ns;
    double sa = 0.0, sb = 0.0;
    for (int it = 0;; ++it) {
        bool ready = true;
        unsigned long long va = 0ull, vb = 0ull;
        if (lane < ncl) {
            ld_relaxed_v2(buf + 2 * static_cast<long long>(lane) * C, va, vb);
            ready = ((va >> 63) == phase) && ((vb >> 63) == phase);
        }
        if (__all_sync(kFull, ready)) {
            if (lane < ncl) {
                sa = __longlong_as_double(static_cast<long long>(va & 0x7fffffffffffffffull));
                sb = __longlong_as_double(static_cast<long long>(vb & 0x7fffffffffffffffull));
            }
            break;
        }
        int give_up = 0;
        if (lane == 0 && (it & 15) == 15)
            give_up = (ld_relaxed_i32(d.abort_flag) != 0) || (now_ns() > deadline);
        if (__shfl_sync(kFull, give_up, 0)) {
            if (lane == 0) atomicExch(d.abort_flag, 1);
            return false;
        }
    }
    A = __shfl_sync(kFull, warp_tree_sum(sa), 0);
    B = __shfl_sync(kFull, warp_tree_sum(sb), 0);
    return true;
}

// Block reduction of two per-thread partials (exact), then the grid all-reduce by warp 0.
// On return (all threads) sh.G, sh.H hold the grid totals; returns false on abort.
__device__ bool block_grid_reduce(const DevLayout &d, int me, unsigned long long seq, long long timeout_ns,
                                  SharedState &sh, Fx fa, Fx fb, bool bad) {
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    fa = fx_warp_sum(fa);
    fb = fx_warp_sum(fb);
    const int wbad = __any_sync(kFull, bad);
    if (lane == 0) {
        sh.wa[warp] = fa;
        sh.wb[warp] = fb;
        sh.wbad[warp] = wbad;
    }
    __syncthreads();
    if (warp == 0) {
        Fx ta = lane < nwarps ? sh.wa[lane] : fx_zero();
        Fx tb = lane < nwarps ? sh.wb[lane] : fx_zero();
        const bool cb = __any_sync(kFull, lane < nwarps ? sh.wbad[lane] != 0 : false);
        ta = fx_warp_sum(ta);
        tb = fx_warp_sum(tb);
        double ca = fx_to_double(ta), cbv = fx_to_double(tb);
        if (cb) ca = cbv = __longlong_as_double(0x7ff8000000000000ll);
        ca = __shfl_sync(kFull, ca, 0);
        cbv = __shfl_sync(kFull, cbv, 0);
        double At = 0.0, Bt = 0.0;
        const bool ok = grid_allreduce2(d, me, seq, ca, cbv, At, Bt, timeout_ns, true);
        if (lane == 0) {
            sh.ok = ok;
            sh.G = At;
            sh.H = Bt;
        }
    }
    __syncthreads();
    return sh.ok != 0;
}

// ------------------------------------------------------------------ the coordinate step

// FP64 issues at 1/64 of the FP32 rate on this part (a warp's FP64 instruction holds its SM
// partition's unit for about 64 clocks, however many lanes are active), so the helpers below
// keep FP64 instructions off the coordinate path where integer or FP32 work can stand in.

__device__ __forceinline__ bool nan_bits_u(unsigned long long b) { return (b & 0x7fffffffffffffffull) > 0x7ff0000000000000ull; }

// a / b: a reciprocal seed from FP32 (b's leading 24 bits, the hardware's approximate
// reciprocal), one Newton-Raphson refinement of the reciprocal and one correction of the
// quotient, both by FMA (P. Markstein, IBM J. Res. Dev. 34(1), 1990).  Five FP64 operations;
// the seed's error (about 2^-22) squares to about 2^-44 in the reciprocal, and the correction
// leaves the quotient within an ulp (faithful; the correctly rounded one in practice).  |b|
// outside [2^-120, 2^121), |a| outside [2^-900, 2^901), zeros, infinities and NaNs take the
// IEEE division.
__device__ __forceinline__ double quot(double a, double b) {
    const unsigned long long ab = static_cast<unsigned long long>(__double_as_longlong(a));
    const unsigned long long bb = static_cast<unsigned long long>(__double_as_longlong(b));
    const unsigned ea = static_cast<unsigned>((ab >> 52) & 0x7ff), eb = static_cast<unsigned>((bb >> 52) & 0x7ff);
    if (eb - (1023u - 120u) > 240u || ea - (1023u - 900u) > 1800u) return a / b;
    const float bf = __int_as_float(static_cast<int>(((eb - 896u) << 23) | static_cast<unsigned>((bb >> 29) & 0x7fffff)));
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(bf));
    const unsigned rb = static_cast<unsigned>(__float_as_int(rf));
    const double y0 = __longlong_as_double(static_cast<long long>(
        (static_cast<unsigned long long>(((rb >> 23) & 0xffu) + 896u) << 52) |
        (static_cast<unsigned long long>(rb & 0x7fffffu) << 29) | (bb & 0x8000000000000000ull)));
    const double e = fma(-b, y0, 1.0);
    const double y1 = fma(y0, e, y0);
    const double q0 = a * y1;
    const double r = fma(-b, q0, a);
    return fma(r, y1, q0);
}

// An unsigned 32-bit integer as a double, assembled from its bits (exact).
__device__ __forceinline__ double u32_to_double(unsigned v) {
    if (v == 0u) return 0.0;
    const int e = 31 - __clz(v);
    return __longlong_as_double(static_cast<long long>((static_cast<unsigned long long>(1023 + e) << 52) |
                                                       ((static_cast<unsigned long long>(v) << (52 - e)) & 0xfffffffffffffull)));
}

// The Genkin trust radius after a step: max(2 |db|, t / 2) (t > 0), exact, by bit patterns;
// radii within a factor 2 of the subnormal range take the FP64 expression.
__device__ __forceinline__ double trust_update(double db, double t) {
    const unsigned long long a = static_cast<unsigned long long>(__double_as_longlong(db)) & 0x7fffffffffffffffull;
    const unsigned long long tb = static_cast<unsigned long long>(__double_as_longlong(t));
    if ((tb >> 52) - 2ull > 0x7fcull || (a >> 52) >= 0x7feull) return fmax(2.0 * fabs(db), 0.5 * t);
    const unsigned long long a2 = a == 0ull ? 0ull : ((a >> 52) == 0ull ? (a << 1) : a + (1ull << 52));
    const unsigned long long t2 = tb - (1ull << 52);
    return __longlong_as_double(static_cast<long long>(a2 > t2 ? a2 : t2));
}

// Newton step of Eq. 4 under the prior of Eq. 3, clamped to the Genkin trust region (one
// lane).  q = -h >= 0.  Laplace: soft threshold at 0, and a step that would change the sign
// of a nonzero b stops at 0.  q = 0 with no finite minimiser takes the trust bound and
// raises warning bit 0.  The trust radius itself is updated by the caller.
__device__ double newton_step(double g, double q, double b, const FitParams &p, double trust, int &warn) {
    double dv;
    if (p.prior == 1) {
        dv = quot(fma(-b, p.inv_var, g), q + p.inv_var);
    } else if (p.prior == 2) {
        const double lambda = p.lambda;
        if (q > 0.0) {
            if (b == 0.0) {
                const double gu = g - lambda, gd = g + lambda;
                dv = gu > 0.0 ? quot(gu, q) : (gd < 0.0 ? quot(gd, q) : 0.0);
            } else {
                const double s = b > 0.0 ? 1.0 : -1.0;
                dv = quot(g - lambda * s, q);
                const double nb = b + dv;
                const double ns = nb > 0.0 ? 1.0 : (nb < 0.0 ? -1.0 : 0.0);
                if (ns != s) dv = -b;
            }
        } else if (b == 0.0) {
            if (fabs(g) <= lambda) {
                dv = 0.0;
            } else {
                dv = g > 0.0 ? trust : -trust;
                warn |= 1;
            }
        } else {
            const double s = b > 0.0 ? 1.0 : -1.0;
            if (fabs(g) <= lambda) {
                dv = -b;
            } else {
                const double dd = g - lambda * s;
                dv = dd > 0.0 ? trust : (dd < 0.0 ? -trust : 0.0);
                const double nb = b + dv;
                const double ns = nb > 0.0 ? 1.0 : (nb < 0.0 ? -1.0 : 0.0);
                if (ns != s) dv = -b;
                warn |= 1;
            }
        }
    } else {
        if (q > 0.0) {
            dv = quot(g, q);
        } else if (g != 0.0) {
            dv = g > 0.0 ? trust : -trust;
            warn |= 1;
        } else {
            dv = 0.0;
        }
    }
    // clamp to [-trust, trust] by bit patterns (trust >= 0; NaN goes to -trust, as fmin/fmax do)
    const unsigned long long db = static_cast<unsigned long long>(__double_as_longlong(dv));
    const unsigned long long tb = static_cast<unsigned long long>(__double_as_longlong(trust));
    if ((db & 0x7fffffffffffffffull) > tb)
        dv = __longlong_as_double(static_cast<long long>(tb | (nan_bits_u(db) ? 0x8000000000000000ull : (db & 0x8000000000000000ull))));
    return dv;
}

// ---- e^x and e^x - 1 for the coordinate step (on every coordinate's critical path).
// |x| < 2^-10: e^x - 1 from its Taylor series to x^5 (the next term is below 2^-59 relative),
// e^x = 1 + that.  Otherwise Tang's table-driven method (P. T. P. Tang, ACM TOMS 15(2), 1989):
// x = (32 m + j) ln2/32 + r with |r| <= ln2/64, e^x = 2^m 2^(j/32) e^r, e^r - 1 from its Taylor
// series to r^6 (the next term is below 2^-60 relative).  n = 32 m + j is x 32/ln2 rounded to
// the nearest integer by adding 1.5 2^52 in one FMA (the sum's low word holds n); 2^m goes into
// the table value's exponent field.  Table: 2^(j/32) rounded to the nearest double (from the
// exponential series at 60 digits); ln2/32 split so that n ln2/32 is exact in two parts for
// |n| < 2^15.  |x| >= 700 (and NaN) go to exp().
__constant__ double c_exp2_j32[32] = {
    0x1.0000000000000p+0, 0x1.059b0d3158574p+0, 0x1.0b5586cf9890fp+0, 0x1.11301d0125b51p+0,
    0x1.172b83c7d517bp+0, 0x1.1d4873168b9aap+0, 0x1.2387a6e756238p+0, 0x1.29e9df51fdee1p+0,
    0x1.306fe0a31b715p+0, 0x1.371a7373aa9cbp+0, 0x1.3dea64c123422p+0, 0x1.44e086061892dp+0,
    0x1.4bfdad5362a27p+0, 0x1.5342b569d4f82p+0, 0x1.5ab07dd485429p+0, 0x1.6247eb03a5585p+0,
    0x1.6a09e667f3bcdp+0, 0x1.71f75e8ec5f74p+0, 0x1.7a11473eb0187p+0, 0x1.82589994cce13p+0,
    0x1.8ace5422aa0dbp+0, 0x1.93737b0cdc5e5p+0, 0x1.9c49182a3f090p+0, 0x1.a5503b23e255dp+0,
    0x1.ae89f995ad3adp+0, 0x1.b7f76f2fb5e47p+0, 0x1.c199bdd85529cp+0, 0x1.cb720dcef9069p+0,
    0x1.d5818dcfba487p+0, 0x1.dfc97337b9b5fp+0, 0x1.ea4afa2a490dap+0, 0x1.f50765b6e4540p+0};

struct ExpStep {
    double r;     // e^x
    double em1;   // e^x - 1
};

__device__ __forceinline__ ExpStep exp_step(double x) {
    const unsigned long long ax = static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7fffffffffffffffull;
    if (ax < 0x3f50000000000000ull) {                // |x| < 2^-10
        double p = fma(x, 1.0 / 120.0, 1.0 / 24.0);
        p = fma(x, p, 1.0 / 6.0);
        p = fma(x, p, 0.5);
        const double em1 = fma(x * x, p, x);
        return ExpStep{1.0 + em1, em1};
    }
    if (ax >= 0x4085e00000000000ull) {               // |x| >= 700, inf, NaN
        const double r = exp(x);
        return ExpStep{r, r - 1.0};
    }
    constexpr double kInvL = 0x1.71547652b82fep+5;   // 32 / ln 2
    constexpr double kL1 = 0x1.62e42fefa0000p-6;     // ln2/32, high 38 bits
    constexpr double kL2 = 0x1.cf79abc9e3b3ap-45;    // ln2/32 - kL1
    constexpr double kShift = 0x1.8p52;
    const double sh = fma(x, kInvL, kShift);
    const int ni = static_cast<int>(__double2loint(sh));
    const double n = sh - kShift;
    const double r = fma(-n, kL2, fma(-n, kL1, x));
    const int jj = ni & 31, m = ni >> 5;             // n = 32 m + jj (arithmetic shift: floor)
    double q = fma(r, 1.0 / 720.0, 1.0 / 120.0);
    q = fma(r, q, 1.0 / 24.0);
    q = fma(r, q, 1.0 / 6.0);
    q = fma(r, q, 0.5);
    const double em1r = fma(r * r, q, r);            // e^r - 1
    const double t = __longlong_as_double(__double_as_longlong(c_exp2_j32[jj]) + (static_cast<long long>(m) << 52));
    const double e = fma(t, em1r, t);
    return ExpStep{e, e - 1.0};
}

// Classifications by bit pattern (integer ops; an FP64 compare costs as much as an FP64 add).
__device__ __forceinline__ bool nan_bits(double v) {
    return (static_cast<unsigned long long>(__double_as_longlong(v)) & 0x7fffffffffffffffull) > 0x7ff0000000000000ull;
}
__device__ __forceinline__ bool nonfinite_bits(double v) {
    return (static_cast<unsigned long long>(__double_as_longlong(v)) & 0x7ff0000000000000ull) == 0x7ff0000000000000ull;
}

// W_i from one segment, with the partials of Eqs. 7 and 9.  W_i is a share of D_i; rounding
// in the incremental D can push it an ulp past 1, so it is clamped (by its bit pattern).
__device__ __forceinline__ void segment_terms(double num, double Dv, int nv, double &gl, double &hl, bool &bad) {
    const unsigned long long bd = static_cast<unsigned long long>(__double_as_longlong(Dv));
    const unsigned long long bn = static_cast<unsigned long long>(__double_as_longlong(num));
    if (bd == 0ull || bd >= 0x7ff0000000000000ull || bn >= 0x7ff0000000000000ull) bad = true;
    double w = quot(num, Dv);
    if (static_cast<unsigned long long>(__double_as_longlong(w)) > 0x3ff0000000000000ull) w = 1.0;
    gl = u32_to_double(static_cast<unsigned>(nv)) * w;
    hl = fma(-gl, w, gl);                             // gl (1 - w), one rounding
}

// ------------------------------------------------------------------ column phases

// Phase A over a staged slice (everything static already in shared memory).
// The JDS groups g0, g0 + gstep, ... below g1 of one column of the staged slice, whose groups
// start at gbase and segments at sbase, sbase + 32, ... up to send (the whole slice of one column:
// g0 = warp, gstep = warps, gbase = sbase = 0, send = segments).
__device__ void phase_a_staged(const DevLayout &d, const ColDesc &cd, const StageBuf &sb, SmemLayout &sm,
                               int g0, int g1, int gstep, int gbase, int sbase, int send, double &G, double &H,
                               bool &bad) {
    const int lane = threadIdx.x & 31;
    const int2 *sseg = sb.segs + cd.seg_off;
    const int32_t *srow = sb.rows + cd.row_off;
    const long long *sgrp = sb.grp + cd.grp_off;
    bool first = true;
    for (int g = g0; g < g1; g += gstep) {
        const int si = sbase + 32 * (g - gbase) + lane;
        const bool valid = si < send;
        const int2 sg = valid ? sseg[si] : make_int2(0, 0);
        const double Dv = valid ? ld_state(d.D + sg.x) : 1.0;
        const int nv = valid ? d.nev[sg.x] : 0;
        int base = static_cast<int>(sgrp[g] - cd.row0);
        const int maxlen = __shfl_sync(kFull, sg.y, 0);  // segments are sorted longest first
        double num = 0.0;
        // one batch of diagonals; the first batch's first diagonal starts the sums (no FP64 add)
        auto batch = [&](int t0, bool init) {
            int pos[kBatch];
            int32_t k[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const bool act = sg.y > t0 + u;
                const unsigned m = __ballot_sync(kFull, act);
                pos[u] = act ? base + lane : -1;
                k[u] = act ? srow[base + lane] : -1;
                base += __popc(m);
            }
            double e[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) e[u] = k[u] >= 0 ? ld_state(d.E + k[u]) : 0.0;
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                if (t0 + u < maxlen) {       // warp-uniform: skip the FP64 add on empty diagonals
                    if (k[u] >= 0) {
                        if (init && u == 0) num = e[u];
                        else num += e[u];
                        sm.wide.est[pos[u]] = e[u];
                    }
                }
            }
        };
        batch(0, true);
        for (int t0 = kBatch; t0 < maxlen; t0 += kBatch) batch(t0, false);
        double gl = 0.0, hl = 0.0;
        if (valid) {
            segment_terms(num, Dv, nv, gl, hl, bad);
            sm.wide.seg_stash[si] = make_double2(num, Dv);
        }
        if (first) {
            G = gl;
            H = hl;
            first = false;
        } else {
            G += gl;
            H += hl;
        }
    }
}

// Phase A over a slice read straight from global memory (slices too big to stage).  Each warp
// walks its groups with a software pipeline: the group descriptors two groups ahead, and the row
// indices of the next group's first kBatch diagonals copied asynchronously into the warp's half
// of a ring in shared memory (the wide buffer, idle while the slice is not staged), so a group's
// E gathers start from rows already on chip instead of behind a dependent load.  Without a ring
// (kRing false: a kernel with no room for it) the rows are read from global memory in place.
template <bool kPipe>
__device__ void phase_a_global(const DevLayout &d, int s, int j, int *ring_all, double &G, double &H, bool &bad,
                               bool stash_e = true) {
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const long long so = static_cast<long long>(s) * (d.J + 1) + j;
    const long long seg0 = d.slice_seg[so], seg1 = d.slice_seg[so + 1];
    const long long grp0 = d.slice_grp[so];
    const int ngrp = static_cast<int>(d.slice_grp[so + 1] - grp0);
    double *stash = d.stash + 2 * static_cast<long long>(s) * d.stash_stride;
    constexpr int kRing = 32 * kBatch;              // rows of a group's first kBatch diagonals, at most
    int *ring = kPipe ? ring_all + warp * (2 * kRing) : nullptr;
    // with the ring (the fit kernel), every gathered E also goes to the slice's E stash at its row
    // position, for phase C
    const long long row0 = d.slice_row[so];
    double *estash = kPipe ? d.estash + static_cast<long long>(s) * d.estash_stride : nullptr;
    auto desc = [&](int g, int2 &sg, long long &base) {
        sg = make_int2(0, 0);
        base = 0;
        if (g < ngrp) {
            const long long si = seg0 + 32 * static_cast<long long>(g) + lane;
            if (si < seg1) sg = ld_static(d.segs + si);
            base = ld_static(d.grp_base + grp0 + g);
        }
    };
    // the rows of a group's first kBatch diagonals are contiguous from its base (segments are
    // longest first, diagonal after diagonal); every lane commits a copy group, empty or not
    auto stage_rows = [&](const int2 &sg, long long base, int half) {
        if (!kPipe) return;
        int R = 0;
#pragma unroll
        for (int u = 0; u < kBatch; ++u) R += __popc(__ballot_sync(kFull, sg.y > u));
        int *dst = ring + half * kRing;
        for (int q = lane; q < R; q += 32) cp_async4(dst + q, d.rows + base + q);
        cp_async_commit();
    };
    bool first = true;
    int2 sg_cur, sg_n1;
    long long base_cur, base_n1;
    desc(warp, sg_cur, base_cur);
    desc(warp + nwarps, sg_n1, base_n1);
    if (warp < ngrp) stage_rows(sg_cur, base_cur, 0);
    int half = 0;
    for (int g = warp; g < ngrp; g += nwarps) {
        const long long si = seg0 + 32 * static_cast<long long>(g) + lane;
        const bool valid = si < seg1;
        const int2 sg = sg_cur;
        const long long gbase = base_cur;
        int2 sg_n2;
        long long base_n2;
        desc(g + 2 * nwarps, sg_n2, base_n2);
        const bool has_next = g + nwarps < ngrp;     // warp-uniform
        if (has_next) stage_rows(sg_n1, base_n1, half ^ 1);
        const double Dv = valid ? ld_state(d.D + sg.x) : 1.0;
        const int nv = valid ? d.nev[sg.x] : 0;
        // this group's rows have landed (every copy group but the newest), for every lane
        if (kPipe) {
            if (has_next) cp_async_wait<1>();
            else cp_async_wait<0>();
            __syncwarp();
        }
        const int *rr = kPipe ? ring + half * kRing : nullptr;
        const int maxlen = __shfl_sync(kFull, sg.y, 0);
        long long base = gbase;
        double num = 0.0;
        auto batch = [&](int t0, bool init, bool staged) {
            int32_t k[kBatch];
            long long pb = base;                      // the batch's first row (stash positions)
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const bool act = sg.y > t0 + u;
                const unsigned m = __ballot_sync(kFull, act);
                k[u] = act ? (staged ? rr[static_cast<int>(base - gbase) + lane] : ld_static(d.rows + base + lane)) : -1;
                base += __popc(m);
            }
            double e[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) e[u] = k[u] >= 0 ? ld_state(d.E + k[u]) : 0.0;
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                if (t0 + u < maxlen) {                // warp-uniform
                    const unsigned m = __ballot_sync(kFull, sg.y > t0 + u);
                    if (k[u] >= 0) {
                        if (init && u == 0) num = e[u];
                        else num += e[u];
                        if (kPipe && stash_e) __stcs(estash + (pb - row0 + lane), e[u]);   // streaming: E stays in L2
                    }
                    pb += __popc(m);
                }
            }
        };
        if (maxlen > 0) batch(0, true, kPipe);
        for (int t0 = kBatch; t0 < maxlen; t0 += kBatch) batch(t0, false, false);
        double gl = 0.0, hl = 0.0;
        if (valid) {
            segment_terms(num, Dv, nv, gl, hl, bad);
            stash[2 * (si - seg0)] = num;
            stash[2 * (si - seg0) + 1] = Dv;
        }
        if (first) {
            G = gl;
            H = hl;
            first = false;
        } else {
            G += gl;
            H += hl;
        }
        if (kPipe) __syncwarp();                      // every lane is done with this half
        sg_cur = sg_n1;
        base_cur = base_n1;
        sg_n1 = sg_n2;
        base_n1 = base_n2;
        half ^= 1;
    }
}

// Phase C over a staged slice: stores only.
__device__ void phase_c_staged(const DevLayout &d, const ColDesc &cd, const StageBuf &sb, const SmemLayout &sm,
                               double r, double em1) {
    const int2 *sseg = sb.segs + cd.seg_off;
    const int32_t *srow = sb.rows + cd.row_off;
    for (int p = threadIdx.x; p < cd.nnz; p += blockDim.x) st_state(d.E + srow[p], sm.wide.est[p] * r);
    for (int si = threadIdx.x; si < cd.nseg; si += blockDim.x) {
        const double2 st = sm.wide.seg_stash[si];
        st_state(d.D + sseg[si].x, fma(em1, st.x, st.y));
    }
}

// Phase C over a global slice.
__device__ void phase_c_global(const DevLayout &d, int s, int j, double r, double em1, bool regather = false) {
    const long long so = static_cast<long long>(s) * (d.J + 1) + j;
    const long long row0 = d.slice_row[so], row1 = d.slice_row[so + 1];
    const long long seg0 = d.slice_seg[so], seg1 = d.slice_seg[so + 1];
    const double *stash = d.stash + 2 * static_cast<long long>(s) * d.stash_stride;
    const long long T = blockDim.x;
    if (regather) {                               // E at the slice's rows again, mostly from L2
        long long p = row0 + threadIdx.x;
        for (; p + 3 * T < row1; p += 4 * T) {
            int32_t k[4];
            double e[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) k[u] = ld_static(d.rows + p + u * T);
#pragma unroll
            for (int u = 0; u < 4; ++u) e[u] = ld_state(d.E + k[u]);
#pragma unroll
            for (int u = 0; u < 4; ++u) st_state(d.E + k[u], e[u] * r);
        }
        for (; p < row1; p += T) {
            const int32_t k = ld_static(d.rows + p);
            st_state(d.E + k, ld_state(d.E + k) * r);
        }
        for (long long si = seg0 + threadIdx.x; si < seg1; si += T) {
            const double num = stash[2 * (si - seg0)], Dv = stash[2 * (si - seg0) + 1];
            st_state(d.D + ld_static(d.segs + si).x, fma(em1, num, Dv));
        }
        return;
    }
    // E as phase A gathered it, at each row's position in the slice (coalesced, no gather)
    const double *estash = d.estash + static_cast<long long>(s) * d.estash_stride - row0;
    long long p = row0 + threadIdx.x;
    for (; p + 3 * T < row1; p += 4 * T) {
        int32_t k[4];
        double e[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            k[u] = d.rows[p + u * T];
            e[u] = __ldcs(estash + p + u * T);   // streaming: read once
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) d.E[k[u]] = e[u] * r;
    }
    for (; p < row1; p += T) d.E[d.rows[p]] = __ldcs(estash + p) * r;
    for (long long si = seg0 + threadIdx.x; si < seg1; si += T) {
        const double num = stash[2 * (si - seg0)], Dv = stash[2 * (si - seg0) + 1];
        d.D[d.segs[si].x] = fma(em1, num, Dv);
    }
}

// ------------------------------------------------------------------ FP32 column phases
//
// FP32 mode (the single-precision variant): E in FP32, each segment's numerator a Kahan
// (compensated) FP32 sum, D_i an FP32 (hi, lo) pair updated with an error-free two-sum, W_i and
// its two terms in FP32; each thread's per-subject terms are summed exactly in fixed point and
// rounded once to FP64, then enter the FP64 sums of the coordinate path.  The scalar step stays
// in FP64.

// Exact conversion of a finite non-negative float below 2^60 (see fx_from_double).
__device__ __forceinline__ Fx fx_from_float(float v, bool &bad) {
    const unsigned b = __float_as_uint(v);
    const int e = static_cast<int>((b >> 23) & 0xff);
    Fx r = fx_zero();
    if ((b >> 31) && b != 0x80000000u) {
        bad = true;
        return r;
    }
    if (e == 0) return r;
    if (e >= 127 + 60) {
        bad = true;
        return r;
    }
    const unsigned long long m = (b & 0x7fffffu) | 0x800000u;
    const int sh = e - 150 + kFrac;              // v = m * 2^(e - 150)
    if (sh < 0) {
        if (sh > -64) r.w0 = m >> (-sh);
        return r;
    }
    const int q = sh >> 6, rm = sh & 63;
    const unsigned long long lo = m << rm;
    const unsigned long long hi = rm ? (m >> (64 - rm)) : 0ull;
    if (q == 0) {
        r.w0 = lo;
        r.w1 = hi;
    } else if (q == 1) {
        r.w1 = lo;
        r.w2 = hi;
    } else {
        r.w2 = lo;
    }
    return r;
}

// Compensated (Kahan) accumulation of one FP32 term.
__device__ __forceinline__ void kahan_add(float &sum, float &comp, float x) {
    const float y = x - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

// (hi, lo) + x with an error-free two-sum, renormalised.
__device__ __forceinline__ float2 pair_add(float2 d, float x) {
    const float s = d.x + x;
    const float bp = s - d.x;
    const float err = (d.x - (s - bp)) + (x - bp);
    const float lo = d.y + err;
    const float hi = s + lo;
    return make_float2(hi, lo - (hi - s));
}

__device__ __forceinline__ void segment_terms32(float num, float Dhi, int nv, Fx &ga, Fx &ha, bool &bad) {
    const unsigned bd = __float_as_uint(Dhi), bn = __float_as_uint(num);
    if (bd == 0u || bd >= 0x7f800000u || bn >= 0x7f800000u) bad = true;
    float w = num / Dhi;
    if (__float_as_uint(w) > 0x3f800000u) w = 1.0f;
    const float gl = static_cast<float>(nv) * w;
    const float hl = gl * (1.0f - w);
    ga = fx_add(ga, fx_from_float(gl, bad));
    ha = fx_add(ha, fx_from_float(hl, bad));
}

__device__ void phase_a_staged32(const DevLayout &d, const ColDesc &cd, const StageBuf &sb, SmemLayout &sm,
                                 Fx &ga, Fx &ha, bool &bad) {
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const int2 *sseg = sb.segs + cd.seg_off;
    const int32_t *srow = sb.rows + cd.row_off;
    const long long *sgrp = sb.grp + cd.grp_off;
    float *est = reinterpret_cast<float *>(sm.wide.est);
    float4 *stash = reinterpret_cast<float4 *>(sm.wide.seg_stash);
    for (int g = warp; g < cd.ngrp; g += nwarps) {
        const int si = 32 * g + lane;
        const bool valid = si < cd.nseg;
        const int2 sg = valid ? sseg[si] : make_int2(0, 0);
        const float2 Dv = valid ? d.D32[sg.x] : make_float2(1.0f, 0.0f);
        const int nv = valid ? d.nev[sg.x] : 0;
        int base = static_cast<int>(sgrp[g] - cd.row0);
        const int maxlen = __shfl_sync(kFull, sg.y, 0);
        float sum = 0.0f, comp = 0.0f;
        for (int t0 = 0; t0 < maxlen; t0 += kBatch) {
            int pos[kBatch];
            int32_t k[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const bool act = sg.y > t0 + u;
                const unsigned m = __ballot_sync(kFull, act);
                pos[u] = act ? base + lane : -1;
                k[u] = act ? srow[base + lane] : -1;
                base += __popc(m);
            }
            float e[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) e[u] = k[u] >= 0 ? d.E32[k[u]] : 0.0f;
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                if (k[u] >= 0) {
                    kahan_add(sum, comp, e[u]);
                    est[pos[u]] = e[u];
                }
            }
        }
        if (valid) {
            const float num = sum - comp;
            segment_terms32(num, Dv.x, nv, ga, ha, bad);
            stash[si] = make_float4(num, Dv.x, Dv.y, 0.0f);
        }
    }
}

// The FP32 counterpart of phase_a_global<true>: the same per-warp pipeline (descriptors two groups
// ahead, the next group's first rows copied into the warp's ring), and every gathered E32 kept in
// the slice's E stash (as floats) for phase C.
__device__ void phase_a_global32(const DevLayout &d, int s, int j, int *ring_all, Fx &ga, Fx &ha, bool &bad) {
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const long long so = static_cast<long long>(s) * (d.J + 1) + j;
    const long long seg0 = d.slice_seg[so], seg1 = d.slice_seg[so + 1];
    const long long grp0 = d.slice_grp[so];
    const int ngrp = static_cast<int>(d.slice_grp[so + 1] - grp0);
    float4 *stash = reinterpret_cast<float4 *>(d.stash + 2 * static_cast<long long>(s) * d.stash_stride);
    constexpr int kRing = 32 * kBatch;
    int *ring = ring_all + warp * (2 * kRing);
    const long long row0 = d.slice_row[so];
    float *estash = reinterpret_cast<float *>(d.estash + static_cast<long long>(s) * d.estash_stride);
    auto desc = [&](int g, int2 &sg, long long &base) {
        sg = make_int2(0, 0);
        base = 0;
        if (g < ngrp) {
            const long long si = seg0 + 32 * static_cast<long long>(g) + lane;
            if (si < seg1) sg = d.segs[si];
            base = d.grp_base[grp0 + g];
        }
    };
    auto stage_rows = [&](const int2 &sg, long long base, int half) {
        int R = 0;
#pragma unroll
        for (int u = 0; u < kBatch; ++u) R += __popc(__ballot_sync(kFull, sg.y > u));
        int *dst = ring + half * kRing;
        for (int q = lane; q < R; q += 32) cp_async4(dst + q, d.rows + base + q);
        cp_async_commit();
    };
    int2 sg_cur, sg_n1;
    long long base_cur, base_n1;
    desc(warp, sg_cur, base_cur);
    desc(warp + nwarps, sg_n1, base_n1);
    if (warp < ngrp) stage_rows(sg_cur, base_cur, 0);
    int half = 0;
    for (int g = warp; g < ngrp; g += nwarps) {
        const long long si = seg0 + 32 * static_cast<long long>(g) + lane;
        const bool valid = si < seg1;
        const int2 sg = sg_cur;
        const long long gbase = base_cur;
        int2 sg_n2;
        long long base_n2;
        desc(g + 2 * nwarps, sg_n2, base_n2);
        const bool has_next = g + nwarps < ngrp;     // warp-uniform
        if (has_next) stage_rows(sg_n1, base_n1, half ^ 1);
        const float2 Dv = valid ? d.D32[sg.x] : make_float2(1.0f, 0.0f);
        const int nv = valid ? d.nev[sg.x] : 0;
        if (has_next) cp_async_wait<1>();
        else cp_async_wait<0>();
        __syncwarp();
        const int *rr = ring + half * kRing;
        const int maxlen = __shfl_sync(kFull, sg.y, 0);
        long long base = gbase;
        float sum = 0.0f, comp = 0.0f;
        for (int t0 = 0; t0 < maxlen; t0 += kBatch) {
            const bool staged = t0 == 0;
            int32_t k[kBatch];
            long long pb = base;
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const bool act = sg.y > t0 + u;
                const unsigned m = __ballot_sync(kFull, act);
                k[u] = act ? (staged ? rr[static_cast<int>(base - gbase) + lane] : d.rows[base + lane]) : -1;
                base += __popc(m);
            }
            float e[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) e[u] = k[u] >= 0 ? d.E32[k[u]] : 0.0f;
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                if (t0 + u < maxlen) {                // warp-uniform
                    const unsigned m = __ballot_sync(kFull, sg.y > t0 + u);
                    if (k[u] >= 0) {
                        kahan_add(sum, comp, e[u]);
                        __stcs(estash + (pb - row0 + lane), e[u]);
                    }
                    pb += __popc(m);
                }
            }
        }
        if (valid) {
            const float num = sum - comp;
            segment_terms32(num, Dv.x, nv, ga, ha, bad);
            stash[si - seg0] = make_float4(num, Dv.x, Dv.y, 0.0f);
        }
        __syncwarp();                                 // every lane is done with this half
        sg_cur = sg_n1;
        base_cur = base_n1;
        sg_n1 = sg_n2;
        base_n1 = base_n2;
        half ^= 1;
    }
}

__device__ void phase_c_staged32(const DevLayout &d, const ColDesc &cd, const StageBuf &sb, const SmemLayout &sm,
                                 float r, float em1) {
    const int2 *sseg = sb.segs + cd.seg_off;
    const int32_t *srow = sb.rows + cd.row_off;
    const float *est = reinterpret_cast<const float *>(sm.wide.est);
    const float4 *stash = reinterpret_cast<const float4 *>(sm.wide.seg_stash);
    for (int p = threadIdx.x; p < cd.nnz; p += blockDim.x) d.E32[srow[p]] = est[p] * r;
    for (int si = threadIdx.x; si < cd.nseg; si += blockDim.x) {
        const float4 st = stash[si];
        d.D32[sseg[si].x] = pair_add(make_float2(st.y, st.z), em1 * st.x);
    }
}

__device__ void phase_c_global32(const DevLayout &d, int s, int j, float r, float em1) {
    const long long so = static_cast<long long>(s) * (d.J + 1) + j;
    const long long row0 = d.slice_row[so], row1 = d.slice_row[so + 1];
    const long long seg0 = d.slice_seg[so], seg1 = d.slice_seg[so + 1];
    const float4 *stash = reinterpret_cast<const float4 *>(d.stash + 2 * static_cast<long long>(s) * d.stash_stride);
    // E32 as phase A gathered it, at each row's position in the slice
    const float *estash = reinterpret_cast<const float *>(d.estash + static_cast<long long>(s) * d.estash_stride) - row0;
    const long long T = blockDim.x;
    long long p = row0 + threadIdx.x;
    for (; p + 3 * T < row1; p += 4 * T) {
        int32_t k[4];
        float e[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            k[u] = d.rows[p + u * T];
            e[u] = __ldcs(estash + p + u * T);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) d.E32[k[u]] = e[u] * r;
    }
    for (; p < row1; p += T) d.E32[d.rows[p]] = __ldcs(estash + p) * r;
    for (long long si = seg0 + threadIdx.x; si < seg1; si += T) {
        const float4 st = stash[si - seg0];
        d.D32[d.segs[si].x] = pair_add(make_float2(st.y, st.z), em1 * st.x);
    }
}

__device__ void prefetch_staged_state32(const DevLayout &d, const ColDesc &nd, const StageBuf &sb, uint64_t *bar,
                                        uint32_t parity) {
    if (!mbar_wait(bar, parity, 20000)) return;
    const int t = threadIdx.x - 32, T = blockDim.x - 32;
    const int32_t *srow = sb.rows + nd.row_off;
    const int2 *sseg = sb.segs + nd.seg_off;
    for (int p = t; p < nd.nnz; p += T) prefetch_l1(d.E32 + srow[p]);
    for (int si = t; si < nd.nseg; si += T) {
        const int i = sseg[si].x;
        prefetch_l1(d.D32 + i);
        prefetch_l1(d.nev + i);
    }
}

// D_i from E in FP32 with compensation, and the exact sums of the positive and negative parts
// of n_i log D_i (FP32 log: the FP32 phase only needs the log-posterior to stop on).
__device__ bool refresh_and_reduce32(const DevLayout &d, int s, unsigned long long seq, long long timeout_ns,
                                     SharedState &sh) {
    const long long p0 = d.shard_pat[s], p1 = d.shard_pat[s + 1];
    Fx fp = fx_zero(), fn = fx_zero();
    bool bad = false;
    for (long long i = p0 + threadIdx.x; i < p1; i += blockDim.x) {
        float sum = 0.0f, comp = 0.0f;
        for (long long k = d.pat_ptr[i]; k < d.pat_ptr[i + 1]; ++k) kahan_add(sum, comp, d.E32[k]);
        const float hi = sum - comp;
        const float lo = -comp - (hi - sum);
        d.D32[i] = make_float2(hi, lo);
        const float t = static_cast<float>(d.nev[i]) * logf(hi);
        if (t >= 0.0f) fp = fx_add(fp, fx_from_float(t, bad));
        else if (t < 0.0f) fn = fx_add(fn, fx_from_float(-t, bad));
        else bad = true;
    }
    return block_grid_reduce(d, s, seq, timeout_ns, sh, fp, fn, bad);
}

// ------------------------------------------------------------------ staging

struct SliceBounds {
    long long seg0, seg1, row0, row1, grp0, grp1;
    int cl;                    // 1: a slice of the cluster partition (cslice_*, crows, csegs, cgrp_base)
    int m;                     // cluster slices: the group's columns (their slices are adjacent)
    long long so0;             // cluster slices: index of the group's first slice in cslice_*
};

__device__ __forceinline__ SliceBounds load_bounds(const DevLayout &d, int s, int j) {
    const long long so = static_cast<long long>(s) * (d.J + 1) + j;
    SliceBounds b;
    b.seg0 = d.slice_seg[so];
    b.seg1 = d.slice_seg[so + 1];
    b.row0 = d.slice_row[so];
    b.row1 = d.slice_row[so + 1];
    b.grp0 = d.slice_grp[so];
    b.grp1 = d.slice_grp[so + 1];
    b.cl = 0;
    return b;
}

// Slices (c, j) .. (c, j + m - 1) of the cluster partition (c < C): a cluster group, one range.
__device__ __forceinline__ SliceBounds load_bounds_c(const DevLayout &d, int c, int j, int m) {
    const long long so = static_cast<long long>(c) * (d.J + 1) + j;
    SliceBounds b;
    b.seg0 = d.cslice_seg[so];
    b.seg1 = d.cslice_seg[so + m];
    b.row0 = d.cslice_row[so];
    b.row1 = d.cslice_row[so + m];
    b.grp0 = d.cslice_grp[so];
    b.grp1 = d.cslice_grp[so + m];
    b.cl = 1;
    b.m = m;
    b.so0 = so;
    return b;
}

// Thread 0: describe slice `b` in desc[buf] and, if it fits, start its bulk copies.
// Returns whether an mbarrier arrival (with its copies) was issued.
__device__ bool issue_stage(const DevLayout &d, const SliceBounds &b, SmemLayout &sm, SharedState &sh, int buf) {
    ColDesc &cd = sh.desc[buf];
    cd.seg0 = b.seg0;
    cd.row0 = b.row0;
    cd.grp0 = b.grp0;
    cd.nseg = static_cast<int>(b.seg1 - b.seg0);
    cd.nnz = static_cast<int>(b.row1 - b.row0);
    cd.ngrp = static_cast<int>(b.grp1 - b.grp0);
    cd.staged = (cd.nseg <= kSegCap && cd.nnz <= kRowCap) ? 1 : 0;
    cd.seg_off = cd.row_off = cd.grp_off = 0;
    cd.cl = b.cl;
    cd.gm = 1;
    if (b.cl) {
        GroupOffs &go = sh.gofs[buf];
        cd.gm = b.m;
        for (int t = 0; t <= b.m; ++t) {
            go.goff[t] = static_cast<int>(d.cslice_grp[b.so0 + t] - b.grp0);
            go.soff[t] = static_cast<int>(d.cslice_seg[b.so0 + t] - b.seg0);
            go.roff[t] = static_cast<int>(d.cslice_row[b.so0 + t] - b.row0);
        }
    }
    if (!cd.staged) return false;
    const int2 *asegs = b.cl ? d.csegs : d.segs;
    const int32_t *arows = b.cl ? d.crows : d.rows;
    const int64_t *agrp = b.cl ? d.cgrp_base : d.grp_base;
    StageBuf &st = sm.stage[buf];
    uint32_t total = 0;
    const char *gs = nullptr, *gr = nullptr, *gg = nullptr;
    uint32_t ns = 0, nr = 0, ng = 0;
    if (cd.nseg > 0) {
        const long long a0 = (8 * b.seg0) & ~15ll, a1 = (8 * b.seg1 + 15) & ~15ll;
        gs = reinterpret_cast<const char *>(asegs) + a0;
        ns = static_cast<uint32_t>(a1 - a0);
        cd.seg_off = static_cast<int>((8 * b.seg0 - a0) / 8);
        const long long r0 = (4 * b.row0) & ~15ll, r1 = (4 * b.row1 + 15) & ~15ll;
        gr = reinterpret_cast<const char *>(arows) + r0;
        nr = static_cast<uint32_t>(r1 - r0);
        cd.row_off = static_cast<int>((4 * b.row0 - r0) / 4);
        const long long g0 = (8 * b.grp0) & ~15ll, g1 = (8 * b.grp1 + 15) & ~15ll;
        gg = reinterpret_cast<const char *>(agrp) + g0;
        ng = static_cast<uint32_t>(g1 - g0);
        cd.grp_off = static_cast<int>((8 * b.grp0 - g0) / 8);
        total = ns + nr + ng;
    }
    fence_proxy_async();
    mbar_arrive_expect_tx(&sh.bar[buf], total);
    if (ns) bulk_g2s(st.segs, gs, ns, &sh.bar[buf]);
    if (nr) bulk_g2s(st.rows, gr, nr, &sh.bar[buf]);
    if (ng) bulk_g2s(st.grp, gg, ng, &sh.bar[buf]);
    return true;
}

// Warps other than warp 0, while warp 0 runs the grid all-reduce: once the next column's
// static slice has landed, pull the E, D and n_i lines it will gather into L1.  Only caches
// are touched, so stale data is impossible; the copy wait is short and its failure harmless.
__device__ void prefetch_staged_state(const DevLayout &d, const ColDesc &nd, const StageBuf &sb, uint64_t *bar,
                                      uint32_t parity) {
    if (!mbar_wait(bar, parity, 20000)) return;
    const int t = threadIdx.x - 32, T = blockDim.x - 32;
    const int32_t *srow = sb.rows + nd.row_off;
    const int2 *sseg = sb.segs + nd.seg_off;
    for (int p = t; p < nd.nnz; p += T) prefetch_l1(d.E + srow[p]);
    for (int si = t; si < nd.nseg; si += T) {
        const int i = sseg[si].x;
        prefetch_l1(d.D + i);
        prefetch_l1(d.nev + i);
    }
}

// ------------------------------------------------------------------ end of cycle

// Recompute D_i = sum_{k in i} E_k on this CTA's subjects and all-reduce the positive and
// negative parts of sum_i n_i log D_i (into sh.G, sh.H).
__device__ bool refresh_and_reduce(const DevLayout &d, int s, unsigned long long seq, long long timeout_ns,
                                   SharedState &sh) {
    const long long p0 = d.shard_pat[s], p1 = d.shard_pat[s + 1];
    double pos = 0.0, neg = 0.0;
    bool bad = false;
    for (long long i = p0 + threadIdx.x; i < p1; i += blockDim.x) {
        double Di = 0.0;
        const long long k0 = d.pat_ptr[i], k1 = d.pat_ptr[i + 1];
        long long k = k0;
        for (; k + 3 < k1; k += 4) {
            const double e0 = d.E[k], e1 = d.E[k + 1], e2 = d.E[k + 2], e3 = d.E[k + 3];
            Di += e0;
            Di += e1;
            Di += e2;
            Di += e3;
        }
        for (; k < k1; ++k) Di += d.E[k];
        d.D[i] = Di;
        const double t = static_cast<double>(d.nev[i]) * log(Di);
        if (t >= 0.0) pos += t;
        else if (t < 0.0) neg -= t;
        else bad = true;  // NaN
    }
    const Fx fp = fx_from_double(pos, bad), fn = fx_from_double(neg, bad);
    return block_grid_reduce(d, s, seq, timeout_ns, sh, fp, fn, bad);
}

// sum_j b_j Y'X_j (= Y'Xb) and the prior term, from this CTA's private beta, in j order.
__device__ void beta_terms(const DevLayout &d, int s, const FitParams &p, double &lin, double &logprior) {
    const double *beta = d.beta_priv + static_cast<long long>(s) * d.J;
    double l = 0.0, sq = 0.0, ab = 0.0;
    for (int j = 0; j < d.J; ++j) {
        const double b = beta[j];
        l = fma(b, d.ytx[j], l);
        sq = fma(b, b, sq);
        ab += fabs(b);
    }
    lin = l;
    logprior = p.prior == 1 ? -0.5 * sq * p.inv_var : (p.prior == 2 ? -p.lambda * ab : 0.0);
}

// The staging thread (last warp, lane 0): wait (bounded) for any bulk copy still in flight
// into this CTA's shared memory.
__device__ void drain_stages(SharedState &sh, unsigned pending, unsigned phase_bits, long long timeout_ns) {
    if (threadIdx.x != static_cast<int>(blockDim.x) - 32) return;
    int ok = 1;
    for (int b = 0; b < 2; ++b)
        if ((pending >> b) & 1u) ok &= mbar_wait(&sh.bar[b], (phase_bits >> b) & 1u, timeout_ns) ? 1 : 0;
    sh.drained = ok;
}

// End of a run: publish its status and sequence number to the CTA, and retire the staging
// barriers (when no copy is outstanding) so the next run can initialise them afresh.
__device__ void finish_run(SharedState &sh, int status, unsigned long long seq) {
    if (threadIdx.x == 0) {
        sh.run_status = status;
        sh.run_seq = seq;
    }
    __syncthreads();
    if (threadIdx.x == 0 && sh.drained) {
        mbar_inval(&sh.bar[0]);
        mbar_inval(&sh.bar[1]);
    }
    __syncthreads();
}

// beta_j <- beta_j + db, the trust-region update T_j <- max(2|db|, T_j / 2), and the cycle's sums
// for the log-posterior's linear and prior terms (in column order).
__device__ __forceinline__ void bookkeep(double *beta, double *trust, int j, double b, double t, double y, double db,
                                         double &lin, double &sq, double &ab, long long &nonzero) {
    const double nbj = b + db;
    beta[j] = nbj;
    trust[j] = trust_update(db, t);
    lin = fma(nbj, y, lin);
    sq = fma(nbj, nbj, sq);
    ab += fabs(nbj);
    if (db != 0.0) ++nonzero;
}

// ------------------------------------------------------------------ narrow columns
//
// A column whose subjects are few is run end to end by the team's CTA 0: gather L x exp(Xb) at
// its rows, each subject's numerator (rows ascending), W terms, the exact CTA-level sums, the
// Newton step (Eq. 4 with the prior and the trust region) and the sparse updates of Section 2.3,
// all with block barriers, no grid-wide all-reduce.  The other CTAs wait for the run of narrow
// columns to end.  The arithmetic per subject and per row is the wide path's; the sums are
// the same exact fixed-point sums of per-thread partials.

// Wait (thread 0) until *ctr >= target, acquiring; bounded, honours the abort flag.
__device__ bool wait_counter(const unsigned long long *ctr, unsigned long long target, const int *abort_flag,
                             long long timeout_ns) {
    const long long t0 = now_ns();
    for (unsigned it = 0;; ++it) {
        unsigned long long v;
        asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(ctr) : "memory");
        if (v >= target) return true;
        if ((it & 15u) == 15u) {
            if (*reinterpret_cast<const volatile int *>(abort_flag)) return false;
            if (now_ns() - t0 > timeout_ns) {
                atomicExch(const_cast<int *>(abort_flag), 1);
                return false;
            }
        }
    }
}

// The state wide column j will read on shard s (E at the slice's rows, D at its subjects) into
// L2, spread over nthr threads.
__device__ __forceinline__ void prefetch_slice_state_l2(const DevLayout &d, int s, int j, int t, int nthr) {
    const long long so = static_cast<long long>(s) * (d.J + 1) + j;
    for (long long q = d.slice_row[so] + t; q < d.slice_row[so + 1]; q += nthr) prefetch_l2(d.E + d.rows[q]);
    for (long long si = d.slice_seg[so] + t; si < d.slice_seg[so + 1]; si += nthr) prefetch_l2(d.D + d.segs[si].x);
}

// Narrow columns j0..j1-1 on this CTA (the team's CTA 0), a group at a time: the columns of a
// group touch pairwise disjoint subjects, so each takes its step on its own warps, side by side,
// with the sequential result.  beta / trust: this CTA's copies; every shard's copy of beta_j is
// written too.  Thread 0 carries status, warn, nonzero.
//
// Pipelined: while the groups' first warps take the steps, the other warps gather the next group
// into the other half of the shared buffers: its size and column offsets, per segment the
// subject, rows, mark and n_i, per row its index into E, and the state (E per row; numerator
// and D per segment).  The run's first group is gathered while CTA 0 waits for the other CTAs.
// A gathered segment is used as it is unless the one step that can have changed its subject
// since (its mark, set on the host: a column of the previous group, or the wide column before
// the run) was not zero; then its state is gathered again.  The W terms are formed after that.
// The static part of a group's data (sizes, segment info, row indices); thread t of nthr takes
// segments t, t + nthr, ...
__device__ void narrow_gather_static(const DevLayout &d, int j, int t, int nthr, NarrowBuf &nb) {
    const int m = d.nar_group[j] > 0 ? d.nar_group[j] : 1;
    const long long ga = d.nar_ptr[j], gb = d.nar_ptr[j + m];
    const int nseg = static_cast<int>(gb - ga);
    const int row0 = nseg > 0 ? d.nar_seg[ga].z : 0;
    if (t <= m) {
        if (t == 0) nb.m = m;
        nb.col_off[t] = static_cast<int>(d.nar_ptr[j + t] - ga);
    }
    for (int q = t; q < nseg; q += nthr) {
        const int4 sg = d.nar_seg[ga + q];
        const int r0 = sg.z - row0;
        nb.info[q] = make_int4(sg.x, sg.y | (sg.w << 16), r0, d.nev[sg.x]);
        for (int u = 0; u < sg.y; ++u) nb.rows[r0 + u] = d.nar_row[sg.z + u];
    }
}

// The state part (numerator, D, E per row) for the same segments as narrow_gather_static with
// the same t and nthr; that call's writes must be visible (a barrier since, or this thread's).
__device__ void narrow_gather_state(const DevLayout &d, int t, int nthr, NarrowBuf &nb) {
    const int nseg = nb.col_off[nb.m];
    for (int q = t; q < nseg; q += nthr) {
        const int4 in = nb.info[q];
        const double Dv = d.D[in.x];
        const int len = in.y & 0xffff;
        double num = d.E[nb.rows[in.z]];
        nb.est[in.z] = num;
        for (int u = 1; u < len; ++u) {
            const double e = d.E[nb.rows[in.z + u]];
            nb.est[in.z + u] = e;
            num += e;
        }
        nb.stash[q] = make_double2(num, Dv);
    }
}

// Both parts at once.
__device__ void narrow_gather(const DevLayout &d, int j, int t, int nthr, NarrowBuf &nb) {
    const int m = d.nar_group[j] > 0 ? d.nar_group[j] : 1;
    const long long ga = d.nar_ptr[j], gb = d.nar_ptr[j + m];
    const int nseg = static_cast<int>(gb - ga);
    const int row0 = nseg > 0 ? d.nar_seg[ga].z : 0;
    if (t <= m) {
        if (t == 0) nb.m = m;
        nb.col_off[t] = static_cast<int>(d.nar_ptr[j + t] - ga);
    }
    for (int q = t; q < nseg; q += nthr) {
        const int4 sg = d.nar_seg[ga + q];
        const double Dv = d.D[sg.x];
        const int nv = d.nev[sg.x];
        const int r0 = sg.z - row0;
        int row = d.nar_row[sg.z];                   // every segment has a row
        double num = d.E[row];
        nb.rows[r0] = row;
        nb.est[r0] = num;
        for (int u = 1; u < sg.y; ++u) {
            row = d.nar_row[sg.z + u];
            const double e = d.E[row];
            nb.rows[r0 + u] = row;
            nb.est[r0 + u] = e;
            num += e;
        }
        nb.stash[q] = make_double2(num, Dv);
        nb.info[q] = make_int4(sg.x, sg.y | (sg.w << 16), r0, nv);
    }
}

__device__ void narrow_columns(const DevLayout &d, const FitParams &p, int j0, int j1, SmemLayout &sm,
                               SharedState &sh, double *beta, double *trust, int &status, int &warn,
                               long long &nonzero) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    int half = 1;                                   // the first group is in nar_hi
    for (int j = j0; j < j1;) {
        NarrowBuf &nb = sm.nar(half);
        const int m = nb.m;
        // warps interleaved over the columns (warp w works for column w mod m), so the group's
        // steppers (warps 0..m-1) sit in different SM partitions and their FP64 chains overlap
        const int wpc = nwarps / m;                 // warps per column
        const int c = warp % m;
        const int wi = warp / m;
        const bool mine = wi < wpc;                 // warps past m * wpc are spare
        const int jc = j + (mine ? c : 0);
        if (threadIdx.x == 0) sh.gnumeric = sh.gwarn = sh.gnonzero = 0;
        // the step's operands early, off the critical path
        const bool stepper = mine && wi == 0 && lane == 0;
        double bj = 0.0, tj = 0.0, yj = 0.0;
        if (stepper) {
            bj = beta[jc];
            tj = trust[jc];
            yj = d.ytx[jc];
        }
        double G = 0.0, H = 0.0;
        bool bad = false, first = true;
        int nseg = 0, so = 0;
        if (mine) {
            so = nb.col_off[c];                     // the column's first slot in the group's buffers
            nseg = nb.col_off[c + 1] - so;
            for (int q = wi * 32 + lane; q < nseg; q += wpc * 32) {
                const int4 in = nb.info[so + q];
                const int mark = in.y >> 16;
                // the step this segment waits on: a column of the previous group, or the wide
                // column before the run (sh.db still holds its step)
                const bool moved = mark != 0 && (mark <= kNarrowGroupMax ? sh.gdb[mark - 1] : sh.db) != 0.0;
                double num, Dv;
                if (!moved) {
                    const double2 st = nb.stash[so + q];   // the subject's state is as gathered
                    num = st.x;
                    Dv = st.y;
                } else {
                    Dv = d.D[in.x];
                    const int len = in.y & 0xffff;
                    num = d.E[nb.rows[in.z]];
                    nb.est[in.z] = num;
                    for (int u = 1; u < len; ++u) {
                        const double e = d.E[nb.rows[in.z + u]];
                        nb.est[in.z + u] = e;
                        num += e;
                    }
                    nb.stash[so + q] = make_double2(num, Dv);
                }
                double gl = 0.0, hl = 0.0;
                segment_terms(num, Dv, in.w, gl, hl, bad);
                if (first) {
                    G = gl;
                    H = hl;
                    first = false;
                } else {
                    G += gl;
                    H += hl;
                }
            }
        }
        const Fx fa = fx_warp_sum(fx_from_double(G, bad));
        const Fx fb = fx_warp_sum(fx_from_double(H, bad));
        const int wbad = __any_sync(kFull, bad);
        if (lane == 0) {
            sh.wa[warp] = fa;
            sh.wb[warp] = fb;
            sh.wbad[warp] = wbad;
        }
        __syncthreads();
        if (mine && wi == 0) {
            // the column's sums over its warps, then its step
            Fx ta = lane < wpc ? sh.wa[c + m * lane] : fx_zero();
            Fx tbx = lane < wpc ? sh.wb[c + m * lane] : fx_zero();
            const bool cbad = __any_sync(kFull, lane < wpc ? sh.wbad[c + m * lane] != 0 : false);
            ta = fx_warp_sum(ta);
            tbx = fx_warp_sum(tbx);
            if (lane == 0) {
                double ca = fx_to_double(ta), cb = fx_to_double(tbx);
                if (cbad) ca = cb = __longlong_as_double(0x7ff8000000000000ll);
                const double g = yj - ca, q = cb;
                int wl = 0;
                double db = newton_step(g, q, bj, p, tj, wl), r = 1.0, em1 = 0.0;
                if (nonfinite_bits(db) || nan_bits(g) || nan_bits(q)) {
                    db = 0.0;
                    atomicExch(&sh.gnumeric, 1);
                } else if (db != 0.0) {
                    const ExpStep es = exp_step(db);
                    r = es.r;
                    em1 = es.em1;
                    atomicAdd(&sh.gnonzero, 1);
                }
                if (wl) atomicOr(&sh.gwarn, wl);
                sh.gdb[c] = db;
                sh.gr[c] = r;
                sh.gem1[c] = em1;
                sh.gnbj[c] = bj + db;
                sh.gtrust[c] = trust_update(db, tj);
            }
        } else if (j + m < j1) {
            // the other warps: gather the next group into the other half of the buffers
            narrow_gather(d, j + m, (warp - m) * 32 + lane, (nwarps - m) * 32, sm.nar(half ^ 1));
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (sh.gnumeric) status = kStNumeric;
            warn |= sh.gwarn;
            nonzero += sh.gnonzero;
        }
        if (mine) {
            const double db = sh.gdb[c];
            if (db != 0.0) {
                const double r = sh.gr[c], em1 = sh.gem1[c];
                for (int q = wi * 32 + lane; q < nseg; q += wpc * 32) {
                    const int4 in = nb.info[so + q];
                    const int len = in.y & 0xffff;
                    for (int u = 0; u < len; ++u) d.E[nb.rows[in.z + u]] = nb.est[in.z + u] * r;
                    const double2 st = nb.stash[so + q];
                    d.D[in.x] = fma(em1, st.x, st.y);
                }
            }
            // bookkeeping, and every shard's copy of beta_jc
            const double nbj = sh.gnbj[c];
            if (wi == 0 && lane == 0) {
                beta[jc] = nbj;
                trust[jc] = sh.gtrust[c];
            }
            for (int t = wi * 32 + lane + 1; t < d.S; t += wpc * 32) d.beta_priv[static_cast<long long>(t) * d.J + jc] = nbj;
        }
        half ^= 1;
        j += m;
        __syncthreads();   // E and D as updated are what the next group reads
    }
}

// ------------------------------------------------------------------ cluster groups
//
// A group of m consecutive cluster columns j .. j + m - 1 with pairwise disjoint subjects, taken by
// the C CTAs of the first cluster, CTA c over cluster shard c (its slices of the m columns are one
// staged range).  Neither column reads the E or D another writes, so their steps are taken side by
// side and the result is the sequential one.  Warps are interleaved over the columns (warp w works
// for column w mod m, as in a narrow group).  Per column: phase A of Section 2.3 over its slice
// (gather L x exp(Xb), the segment numerators, the W terms of Eqs. 7-9), the CTA's sums,
// then warp t sends its column's pair to slot [t][c] of every CTA of the cluster by asynchronous
// stores counted on the receiver's mbarrier of this round (r & 1; armed by warp 0 for the C x m
// pairs it receives), waits (bounded) for that phase, adds the C pairs in a fixed order -- every CTA holds
// the same totals -- and lane 0 takes the step of Eq. 4 (prior, trust region) for column j + t.
// Then phase C for every column with db != 0.  A CTA is at most one round ahead of another (the
// round after needs the slower CTA's own pairs), so bytes of round r + 1 only meet the other
// mbarrier, whose phase for round r - 1 is complete; bytes that arrive before the receiver armed
// it leave its byte count negative until it does, which the mbarrier allows.
// Results in sh.gdb / gr / gem1 / gnbj (and sh.gnumeric, sh.gwarn); false on abort.
__device__ bool cluster_group(const DevLayout &d, const FitParams &p, const ColDesc &cd, const GroupOffs &go,
                              const StageBuf &sb, SmemLayout &sm, SharedState &sh, int rank, int j, unsigned round,
                              const double *beta, const double *trust, bool staged_ok, long long timeout_ns) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int m = cd.gm;
    // warps per column (the host keeps m <= warps / 2); the last warp, whose lane 0 is the staging
    // thread with the previous group's bookkeeping to do, takes no column
    const int wpc = (nwarps - 1) / m;
    const int t = warp % m, wi = warp / m;
    const bool mine = wi < wpc;
    if (threadIdx.x == 0) {
        sh.gnumeric = sh.gwarn = 0;
        sh.ok = 1;
    }
    // the stepping lanes' scalars, loaded now so that their latency hides behind phase A
    double bj = 0.0, tj = 0.0, yj = 0.0;
    if (warp < m && lane == 0) {
        bj = beta[j + warp];
        tj = trust[j + warp];
        yj = d.ytx[j + warp];
    }
    double G = 0.0, H = 0.0;
    bool bad = !cd.staged || !staged_ok;          // never unstaged: the host sizes groups to the buffer
    if (!staged_ok && threadIdx.x == 0) atomicExch(d.abort_flag, 1);   // a stage that did not arrive
    if (!bad && mine)
        phase_a_staged(d, cd, sb, sm, go.goff[t] + wi, go.goff[t + 1], wpc, go.goff[t], go.soff[t], go.soff[t + 1], G, H,
                       bad);
    {
        double fa = G, fb = H;
        warp_tree_sum2(fa, fb, bad);
        const int wbad = __any_sync(kFull, bad);
        if (lane == 0) {
            sh.wda[warp] = fa;
            sh.wdb[warp] = fb;
            sh.wbad[warp] = wbad;
        }
    }
    __syncthreads();
    if (warp < m) {
        const int C = d.C;
        const int buf = static_cast<int>(round & 1u);
        const uint32_t parity = (round >> 1) & 1u;
        // this CTA's total for column warp, over that column's warps (a fixed FP64 tree)
        double ca, cb;
        if (wpc == 1) {                 // one warp per column: its sum is the CTA's
            ca = sh.wda[warp];
            cb = sh.wdb[warp];
        } else {
            ca = warp_tree_sum16(lane < wpc ? sh.wda[warp + m * lane] : 0.0);
            cb = warp_tree_sum16(lane < wpc ? sh.wdb[warp + m * lane] : 0.0);
        }
        const bool cbad = __any_sync(kFull, lane < wpc ? sh.wbad[warp + m * lane] != 0 : false);
        if (cbad) ca = cb = __longlong_as_double(0x7ff8000000000000ll);
        ca = __shfl_sync(kFull, ca, 0);
        cb = __shfl_sync(kFull, cb, 0);
        if (warp == 0 && lane == 0) mbar_arrive_expect_tx(&sh.cbar[buf], static_cast<uint32_t>(16 * C * m));
        if (lane < C)
            st_async_f64x2(cluster_addr(&sh.cslot[buf][warp][rank], lane), ca, cb, cluster_addr(&sh.cbar[buf], lane));
        int ok = 1;
        if (!mbar_try_wait(&sh.cbar[buf], parity)) {
            const long long deadline = now_ns() + timeout_ns;
            for (int it = 0;; ++it) {
                if (mbar_try_wait(&sh.cbar[buf], parity)) break;
                if ((it & 31) == 31 && (ld_relaxed_i32(d.abort_flag) != 0 || now_ns() > deadline)) {
                    ok = 0;
                    break;
                }
            }
        }
        if (!__all_sync(kFull, ok)) {
            if (lane == 0) {
                atomicExch(d.abort_flag, 1);
                sh.ok = 0;
            }
        } else {
            // the C CTA totals, added by a fixed FP64 tree over the ranks: lane 0's order of
            // additions is the same in every CTA, so every
            // CTA takes the same step, and it does not depend on when the pairs arrived.  (An exact
            // fixed-point sum here cost about 0.8 us more per group on the critical path.)  A bad
            // total is a NaN, which the tree carries through.
            double At = 0.0, Bt = 0.0;
            if (lane < C) {
                const double2 v = sh.cslot[buf][warp][lane];
                At = v.x;
                Bt = v.y;
            }
            At = warp_tree_sum16(At);
            Bt = warp_tree_sum16(Bt);
            if (lane == 0) {
                const double g = yj - At, q = Bt;
                int wl = 0;
                double db = newton_step(g, q, bj, p, tj, wl), r = 1.0, em1 = 0.0;
                if (nonfinite_bits(db) || nan_bits(g) || nan_bits(q)) {
                    db = 0.0;
                    atomicExch(&sh.gnumeric, 1);
                } else if (db != 0.0) {
                    const ExpStep es = exp_step(db);
                    r = es.r;
                    em1 = es.em1;
                }
                if (wl) atomicOr(&sh.gwarn, wl);
                sh.gdb[warp] = db;
                sh.gr[warp] = r;
                sh.gem1[warp] = em1;
                sh.gnbj[warp] = bj + db;
                sh.gb[warp] = bj;
                sh.gt[warp] = tj;
                sh.gy[warp] = yj;
            }
        }
    }
    __syncthreads();
    if (!sh.ok) return false;
    // phase C: E_k <- E_k e^{db} on the column's rows, D_i <- D_i + (e^{db} - 1) num_i on its subjects
    const int2 *sseg = sb.segs + cd.seg_off;
    const int32_t *srow = sb.rows + cd.row_off;
    for (int c = 0; c < m; ++c) {
        const double db = sh.gdb[c];
        if (db == 0.0) continue;
        const double r = sh.gr[c], em1 = sh.gem1[c];
        for (int q = go.roff[c] + threadIdx.x; q < go.roff[c + 1]; q += blockDim.x) d.E[srow[q]] = sm.wide.est[q] * r;
        for (int q = go.soff[c] + threadIdx.x; q < go.soff[c + 1]; q += blockDim.x) {
            const double2 st = sm.wide.seg_stash[q];
            d.D[sseg[q].x] = fma(em1, st.x, st.y);
        }
    }
    return true;
}

// ------------------------------------------------------------------ kernels

__device__ void init_shard(const DevLayout &d, int s, const double *beta0, bool keep_trust);
__device__ void e_to_f32_shard(const DevLayout &d, int s);

// One fit (Algorithm 1) on the CTA that owns shard `s` of `d` (d.S CTAs take part).  F32
// selects the FP32 mode; the scalar step is FP64 in both.
template <bool F32>
__device__ void run_fit(const DevLayout &d, const FitParams &p, FitOut *out, double *hist, int s, SmemLayout &sm,
                        SharedState &sh) {
    const bool leader = (s == 0) && (threadIdx.x == 0);
    const long long timeout = p.timeout_ns;
    unsigned long long seq = p.seq_src ? *p.seq_src : p.seq0;
    double *beta = d.beta_priv + static_cast<long long>(s) * d.J;
    double *trust = d.trust_priv + static_cast<long long>(s) * d.J;
    const int J = d.J;

    // staging state: pending and nb live in the last warp's lane 0; phase_bits in every thread
    unsigned pending = 0u;      // buffers with an arrival issued and not yet waited for
    unsigned phase_bits = 0u;   // expected parity per buffer
    SliceBounds nb{};           // bounds of the column after the staged one
    int status = kStNotConverged, warn = 0, cycles = 0;
    long long nonzero = 0;
    double P_prev = 0.0, P = 0.0, conv = 0.0, loglik = 0.0, heldout = __longlong_as_double(0x7ff8000000000000ll);
    long long col = 0;          // wide columns processed: stage buffer = col & 1
    // cluster columns (FP64 fits launched in clusters of d.C CTAs): the first cluster's CTAs (s < C)
    // run every column, the cluster columns over subject shards of their own; the other CTAs run
    // the grid columns only and wait while the cluster runs the rest
    const bool use_cluster = !F32 && p.cluster != 0 && d.C > 0 && d.ccls != nullptr;
    const bool in_cluster = use_cluster && s < d.C;
    const bool cl_launch = !F32 && p.cluster != 0 && d.C > 0 && d.S / d.C <= 32;   // launched in clusters of d.C CTAs
    const bool use_narrow = !F32 && !use_cluster && d.narrow != nullptr;
    unsigned cround = 0;             // cluster all-reduce rounds taken (one per cluster column)
    unsigned long long crun = 0;     // cluster runs in this launch
    // the column this CTA takes after j (cyclically), and its slice's bounds
    // (in the first cluster a cluster column here is a group's first column: the group is one unit)
    auto next_col = [&](int j) -> int {
        if (use_narrow) return d.next_wide[j];
        if (use_cluster && !in_cluster) return d.next_grid[j];
        const int jn = j + ((in_cluster && d.ccls[j]) ? d.cgroup[j] : 1);
        return jn < d.J ? jn : 0;
    };
    auto col_bounds = [&](int j) -> SliceBounds {
        return (in_cluster && d.ccls[j]) ? load_bounds_c(d, s, j, d.cgroup[j]) : load_bounds(d, s, j);
    };
    // Genkin's rule (the paper's Section 2.2 criterion): sum_k |d(Xb)_k| / (1 + sum_k |(Xb)_k|) over
    // a cycle, with (Xb)_k = log(E_k / l_k) and d(Xb)_k = log(E_k / E_k at the cycle's start).
    const bool genkin = !F32 && p.tol_mode == 2 && d.E_prev != nullptr;
    unsigned long long run_id = 0;   // narrow runs in this launch
    long long nonzero_nar = 0;       // thread 0 of CTA 0: narrow steps with db != 0

    if (threadIdx.x == 0) {
        if (use_narrow && s == 0) {   // reset before this CTA's first all-reduce arrival
            d.nar_sync[0] = 0ull;
            d.nar_sync[16] = 0ull;
            __threadfence();
        }
        if (use_cluster && s == 0) {
            d.clu_sync[0] = 0ull;
            d.clu_sync[16] = 0ull;
            __threadfence();
        }
        mbar_init(&sh.bar[0], 1);
        mbar_init(&sh.bar[1], 1);
        mbar_init_fence();
        sh.desc[0].staged = 0;
        sh.desc[1].staged = 0;
        sh.nonzero = 0;
        sh.drained = 1;
        sh.nar_pre = -1;
    }
    __syncthreads();
    // staging (copies, pending set, next bounds) belongs to the last warp's lane 0
    if (threadIdx.x == static_cast<int>(blockDim.x) - 32 && J > 0 && p.max_cycles > 0 &&
        (!use_narrow || d.first_wide >= 0) && (!use_cluster || in_cluster || d.first_grid >= 0)) {
        const int j0 = use_narrow ? d.first_wide : (use_cluster && !in_cluster ? d.first_grid : 0);
        const SliceBounds b0 = col_bounds(j0);
        if (issue_stage(d, b0, sm, sh, 0)) pending |= 1u;
        nb = col_bounds(next_col(j0));
    }
    __syncthreads();

    // P at the start point.
    if (!(F32 ? refresh_and_reduce32(d, s, seq++, timeout, sh) : refresh_and_reduce(d, s, seq++, timeout, sh)))
        goto aborted;
    {
        double lin = 0.0, lp = 0.0;
        if (threadIdx.x == 0) beta_terms(d, s, p, lin, lp);
        loglik = lin - (sh.G - sh.H);
        P_prev = loglik + lp;
        P = P_prev;
        if (leader && p.record_history) hist[0] = P_prev;
        if (threadIdx.x == 0) sh.stop = (!(P_prev == P_prev) || isinf(P_prev)) ? kStNumeric : kStNotConverged;
        __syncthreads();
        status = sh.stop;
    }
    if (genkin)
        for (long long k = d.shard_row[s] + threadIdx.x; k < d.shard_row[s + 1]; k += blockDim.x) d.E_prev[k] = d.E[k];
    {
        // Bookkeeping of a finished column (beta, trust radius, the cycle's sums) is done by
        // thread tb at the start of the next column, off the critical path.
        const int tb = blockDim.x - 32;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
        int pend_j = -1;
        double pend_b = 0.0, pend_t = 0.0, pend_y = 0.0, pend_db = 0.0;
        int pend_gj = 0, pend_gm = 0;   // a cluster group awaiting its bookkeeping (its results in sh.g*)
        double lin_c = 0.0, sq_c = 0.0, ab_c = 0.0;
        long long nonzero_tb = 0;
        for (int c = 1; c <= p.max_cycles && status == kStNotConverged; ++c) {
            lin_c = sq_c = ab_c = 0.0;
            for (int j = 0; j < J; ++j, ++col) {
                if (use_narrow && d.narrow[j]) {
                    // a run of narrow columns: CTA 0 runs them, the others wait; then every CTA
                    // adds the run's columns to its cycle sums, in column order
                    int j1 = j + 1;
                    while (j1 < J && d.narrow[j1]) ++j1;
                    ++run_id;
                    __syncthreads();
                    if (s != 0) {
                        if (threadIdx.x == 0) {
                            // after the barrier, thread 0's fence orders the whole CTA's E and D
                            // writes before the arrival (cumulativity)
                            __threadfence();
                            atomicAdd(&d.nar_sync[0], 1ull);
                            sh.ok = wait_counter(&d.nar_sync[16], run_id, d.abort_flag, timeout) ? 1 : 0;
                        } else if (d.first_wide >= 0) {
                            // while CTA 0 runs the narrow columns: the next wide column's state
                            // on this shard into L2
                            const int jw = d.next_wide[j1 - 1];
                            prefetch_slice_state_l2(d, s, jw, threadIdx.x - 1, blockDim.x - 1);
                        }
                        __syncthreads();
                    } else {
                        // while thread 0 waits for the other CTAs, warps 1.. gather the run's first
                        // group: every write before the previous wide column is visible (its
                        // all-reduce was a release/acquire round); what that column itself changes
                        // on other shards, the segments' marks send back for a second read
                        if (threadIdx.x == 0)
                            sh.ok = wait_counter(&d.nar_sync[0], run_id * static_cast<unsigned long long>(d.S - 1),
                                                 d.abort_flag, timeout) ? 1 : 0;
                        else if (warp >= 1) {
                            if (sh.nar_pre == j)
                                narrow_gather_state(d, threadIdx.x - 32, blockDim.x - 32, sm.nar_hi);
                            else
                                narrow_gather(d, j, threadIdx.x - 32, blockDim.x - 32, sm.nar_hi);
                        }
                        __syncthreads();
                        if (sh.ok) {
                            narrow_columns(d, p, j, j1, sm, sh, beta, trust, status, warn, nonzero_nar);
                            __syncthreads();
                            if (threadIdx.x == 0)   // a release after the barrier covers the CTA's writes
                                asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(&d.nar_sync[16]), "l"(run_id)
                                             : "memory");
                        }
                    }
                    if (!sh.ok) goto aborted;
                    if (threadIdx.x == tb) {
                        if (pend_j >= 0) {
                            bookkeep(beta, trust, pend_j, pend_b, pend_t, pend_y, pend_db, lin_c, sq_c, ab_c, nonzero_tb);
                            pend_j = -1;
                        }
                        for (int jj = j; jj < j1; ++jj) {
                            const double b = beta[jj];
                            lin_c = fma(b, d.ytx[jj], lin_c);
                            sq_c = fma(b, b, sq_c);
                            ab_c += fabs(b);
                        }
                    }
                    j = j1 - 1;
                    --col;             // the loop's increments: no wide column was processed
                    continue;
                }
                const bool clcol = use_cluster && d.ccls[j] != 0;   // a cluster column
                if (clcol && !in_cluster) {
                    // a run of cluster columns, taken by the first cluster: arrive (this CTA's writes
                    // released), wait for the run's end (acquire) while the next grid column's state
                    // on this shard goes to L2, then add the run's columns to the cycle sums in column
                    // order (the cluster wrote every shard's copy of their beta)
                    int j1 = j + 1;
                    while (j1 < J && d.ccls[j1]) ++j1;
                    ++crun;
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        __threadfence();
                        atomicAdd(&d.clu_sync[0], 1ull);
                        sh.ok = wait_counter(&d.clu_sync[16], crun * static_cast<unsigned long long>(d.C),
                                             d.abort_flag, timeout) ? 1 : 0;
                    } else if (d.first_grid >= 0) {
                        prefetch_slice_state_l2(d, s, d.next_grid[j1 - 1], threadIdx.x - 1, blockDim.x - 1);
                    }
                    __syncthreads();
                    if (!sh.ok) goto aborted;
                    if (threadIdx.x == tb) {
                        if (pend_j >= 0) {
                            bookkeep(beta, trust, pend_j, pend_b, pend_t, pend_y, pend_db, lin_c, sq_c, ab_c, nonzero_tb);
                            pend_j = -1;
                        }
                        for (int jj = j; jj < j1; ++jj) {
                            const double b = beta[jj];
                            lin_c = fma(b, d.ytx[jj], lin_c);
                            sq_c = fma(b, b, sq_c);
                            ab_c += fabs(b);
                        }
                    }
                    j = j1 - 1;
                    --col;             // the loop's increments: no column was processed here
                    continue;
                }
                const int gm = clcol ? d.cgroup[j] : 1;              // columns taken as one unit
                const bool run_first = clcol && (j == 0 || !d.ccls[j - 1]);
                const bool run_last = clcol && (j + gm == J || !d.ccls[j + gm]);
                if (run_first) {
                    // entering a cluster run: every CTA of the team has arrived after its last grid
                    // column's updates (released), so this CTA may read and write any subject
                    ++crun;
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        __threadfence();
                        atomicAdd(&d.clu_sync[0], 1ull);
                        sh.ok = wait_counter(&d.clu_sync[0], crun * static_cast<unsigned long long>(d.S), d.abort_flag,
                                             timeout) ? 1 : 0;
                    }
                    __syncthreads();
                    if (!sh.ok) goto aborted;
                }
                const int buf = static_cast<int>(col & 1);
                double bj = 0.0, tj = 0.0, yj = 0.0;
                if (threadIdx.x == 0 || threadIdx.x == tb) {
                    bj = beta[j];
                    tj = trust[j];
                    yj = d.ytx[j];
                }
                // desc[buf] was written a column ago and is stable; wait for its copies
                const ColDesc cd = sh.desc[buf];
                bool staged_ok = true;
                if (cd.staged) {
                    staged_ok = mbar_wait(&sh.bar[buf], (phase_bits >> buf) & 1u, timeout);
                    phase_bits ^= 1u << buf;
                    if (threadIdx.x == tb) pending &= ~(1u << buf);
                }
                // a CTA-wide verdict on the copies (buffer buf ^ 1 is free from here on)
                staged_ok = __syncthreads_and(staged_ok) != 0;
                if (threadIdx.x == tb) {
                    // stage the next column, then the deferred bookkeeping of the previous one
                    if (issue_stage(d, nb, sm, sh, buf ^ 1)) pending |= 1u << (buf ^ 1);
                    nb = col_bounds(next_col(next_col(j)));
                    if (pend_j >= 0) {
                        bookkeep(beta, trust, pend_j, pend_b, pend_t, pend_y, pend_db, lin_c, sq_c, ab_c, nonzero_tb);
                        pend_j = -1;
                    }
                    // a cluster group's results stay in sh.g* until the next group's steps, which
                    // come after the barrier that follows phase A, where this thread arrives later
                    for (int t = 0; t < pend_gm; ++t)
                        bookkeep(beta, trust, pend_gj + t, sh.gb[t], sh.gt[t], sh.gy[t], sh.gdb[t], lin_c, sq_c, ab_c,
                                 nonzero_tb);
                    pend_gm = 0;
                }
                if (clcol) {
                    // a cluster group: steps, updates, then the bookkeeping of its columns in order
                    if (!cluster_group(d, p, cd, sh.gofs[buf], sm.stage[buf], sm, sh, s, j, cround, beta, trust, staged_ok,
                                       timeout))
                        goto aborted;
                    ++cround;
                    if (threadIdx.x == 0) {
                        if (sh.gnumeric) status = kStNumeric;
                        warn |= sh.gwarn;
                    }
                    if (threadIdx.x == tb) {   // the bookkeeping waits for the next unit (off this one's path)
                        pend_gj = j;
                        pend_gm = gm;
                    }
                    // the CTAs outside the cluster keep their own copy of beta (for their cycle sums)
                    for (int t = 0; t < gm; ++t) {
                        const double nbj = sh.gnbj[t];
                        for (int q = d.C + s + static_cast<int>(threadIdx.x) * d.C; q < d.S;
                             q += static_cast<int>(blockDim.x) * d.C)
                            d.beta_priv[static_cast<long long>(q) * J + j + t] = nbj;
                    }
                    __syncthreads();   // E and D writes visible to the next unit's reads
                    if (run_last) {
                        // leaving a cluster run: its writes (E, D, every shard's beta) released to the
                        // team, and the other cluster CTAs' writes acquired before the grid columns
                        if (threadIdx.x == 0) {
                            __threadfence();
                            atomicAdd(&d.clu_sync[16], 1ull);
                            sh.ok = wait_counter(&d.clu_sync[16], crun * static_cast<unsigned long long>(d.C),
                                                 d.abort_flag, timeout) ? 1 : 0;
                        }
                        __syncthreads();
                        if (!sh.ok) goto aborted;
                    }
                    j += gm - 1;
                    continue;
                }
                // this thread's partial sums (FP32 mode: its exact sums of FP32 terms, rounded once)
                double G = 0.0, H = 0.0;
                bool bad = false;
                if (cd.staged && !staged_ok) {          // never read a stage that did not arrive
                    bad = true;
                    if (threadIdx.x == 0) atomicExch(d.abort_flag, 1);
                } else if (F32) {
                    Fx ga = fx_zero(), ha = fx_zero();
                    if (cd.staged) phase_a_staged32(d, cd, sm.stage[buf], sm, ga, ha, bad);
                    else phase_a_global32(d, s, j, reinterpret_cast<int *>(&sm.wide), ga, ha, bad);
                    G = fx_to_double(ga);
                    H = fx_to_double(ha);
                } else {
                    if (cd.staged)
                        phase_a_staged(d, cd, sm.stage[buf], sm, warp, cd.ngrp, nwarps, 0, 0, cd.nseg, G, H, bad);
                    else phase_a_global<true>(d, s, j, reinterpret_cast<int *>(&sm.wide), G, H, bad, !p.regather_e);
                }
                // The CTA's total by fixed FP64 trees (each warp's lanes, then the warps' sums in warp
                // order): the same additions in the same order on every launch.  A slice of at most
                // one group lives in warp 0 alone: its warp sum is the CTA's.
                const bool one_warp = cd.staged && cd.ngrp <= 1;
                if (!one_warp) {
                    double fa = G, fb = H;
                    warp_tree_sum2(fa, fb, bad);
                    const int wbad = __any_sync(kFull, bad);
                    if (lane == 0) {
                        sh.wda[warp] = fa;
                        sh.wdb[warp] = fb;
                        sh.wbad[warp] = wbad;
                    }
                    __syncthreads();
                }
                if (warp == 0) {
                    double ca, cb;
                    bool cbad;
                    if (one_warp) {
                        ca = warp_tree_sum(G);
                        cb = warp_tree_sum(H);
                        cbad = __any_sync(kFull, bad);
                    } else {
                        ca = warp_tree_sum16(lane < nwarps ? sh.wda[lane] : 0.0);   // at most 16 warps
                        cb = warp_tree_sum16(lane < nwarps ? sh.wdb[lane] : 0.0);
                        cbad = __any_sync(kFull, lane < nwarps ? sh.wbad[lane] != 0 : false);
                    }
                    if (cbad) ca = cb = __longlong_as_double(0x7ff8000000000000ll);
                    ca = __shfl_sync(kFull, ca, 0);
                    cb = __shfl_sync(kFull, cb, 0);
                    // grid all-reduce, then the step in lane 0 (no extra barrier)
                    double At = 0.0, Bt = 0.0;
                    // before a narrow run, a release/acquire round: CTA 0 then reads every
                    // shard's E and D as of this column's start (the run's first gather)
                    const bool before_run = use_narrow && d.next_wide[j] != (j + 1 < J ? j + 1 : 0);
                    // in a launch in clusters the CTAs of each cluster first meet in distributed
                    // shared memory, and only the clusters' totals go through global memory
                    const bool ok = cl_launch
                                        ? cluster_grid_allreduce2(d, sh, s, s % d.C, cround, seq, ca, cb, At, Bt, timeout)
                                        : grid_allreduce2(d, s, seq, ca, cb, At, Bt, timeout, before_run);
                    if (lane == 0) {
                        double db = 0.0, r = 1.0, em1 = 0.0;
                        if (ok) {
                            const double g = yj - At, q = Bt;
                            db = newton_step(g, q, bj, p, tj, warn);
                            if (nonfinite_bits(db) || nan_bits(g) || nan_bits(q)) {
                                db = 0.0;
                                status = kStNumeric;
                            } else if (db != 0.0) {
                                const ExpStep es = exp_step(db);
                                r = es.r;
                                em1 = es.em1;
                            }
                        }
                        sh.ok = ok;
                        sh.db = db;
                        sh.r = r;
                        sh.em1 = em1;
                    }
                } else {
                    // warps 1..: desc[buf ^ 1] (written by thread tb) is visible after this barrier
                    if (one_warp) named_barrier_all_but_warp0();
                    const ColDesc &nd = sh.desc[buf ^ 1];
                    // no early L1 copies of state that a narrow run, or the other CTAs, will change
                    // first: the next column of this CTA is taken by another team (cluster / grid),
                    // or a cluster run comes between
                    const bool narrow_gap = use_narrow && d.next_wide[j] != (j + 1 < J ? j + 1 : 0);
                    const bool gap = narrow_gap || (in_cluster && (j + 1 >= J || d.ccls[j] != d.ccls[j + 1])) ||
                                     (use_cluster && !in_cluster && d.next_grid[j] != j + 1);
                    if (narrow_gap && s == 0 && j + 1 < J) {
                        // the next narrow run's first group: its static data, while the
                        // all-reduce runs (E and D are read once the other CTAs arrive)
                        narrow_gather_static(d, j + 1, threadIdx.x - 32, blockDim.x - 32, sm.nar_hi);
                        if (threadIdx.x == 32) sh.nar_pre = j + 1;
                    }
                    if (nd.staged && !gap) {
                        if (F32)
                            prefetch_staged_state32(d, nd, sm.stage[buf ^ 1], &sh.bar[buf ^ 1],
                                                    (phase_bits >> (buf ^ 1)) & 1u);
                        else
                            prefetch_staged_state(d, nd, sm.stage[buf ^ 1], &sh.bar[buf ^ 1],
                                                  (phase_bits >> (buf ^ 1)) & 1u);
                    }
                }
                ++seq;
                if (cl_launch) ++cround;
                __syncthreads();
                if (!sh.ok) goto aborted;
                const double db = sh.db;
                if (db != 0.0) {
                    if (F32) {
                        const float r32 = static_cast<float>(sh.r), em32 = static_cast<float>(sh.em1);
                        if (cd.staged) phase_c_staged32(d, cd, sm.stage[buf], sm, r32, em32);
                        else phase_c_global32(d, s, j, r32, em32);
                    } else {
                        if (cd.staged) phase_c_staged(d, cd, sm.stage[buf], sm, sh.r, sh.em1);
                        else phase_c_global(d, s, j, sh.r, sh.em1, p.regather_e != 0);
                    }
                }
                if (threadIdx.x == tb) {
                    pend_j = j;
                    pend_b = bj;
                    pend_t = tj;
                    pend_y = yj;
                    pend_db = db;
                }
                __syncthreads();   // E and D writes visible to the next column's reads
            }
            if (threadIdx.x == tb) {
                if (pend_j >= 0) {
                    bookkeep(beta, trust, pend_j, pend_b, pend_t, pend_y, pend_db, lin_c, sq_c, ab_c, nonzero_tb);
                    pend_j = -1;
                }
                for (int t = 0; t < pend_gm; ++t)
                    bookkeep(beta, trust, pend_gj + t, sh.gb[t], sh.gt[t], sh.gy[t], sh.gdb[t], lin_c, sq_c, ab_c,
                             nonzero_tb);
                pend_gm = 0;
                sh.lin = lin_c;
                sh.sq = sq_c;
                sh.ab = ab_c;
                sh.nonzero = nonzero_tb;
            }
            __syncthreads();
            if (c % (F32 ? kRebuildCycles32 : kRebuildCycles64) == 0 && d.row_ptr) {
                // bound the rounding drift of the multiplicative updates: E from this CTA's beta copy
                // (every copy holds the same beta), then D and P from it below
                init_shard(d, s, beta, true);
                if (F32) e_to_f32_shard(d, s);
            }
            if (!(F32 ? refresh_and_reduce32(d, s, seq++, timeout, sh) : refresh_and_reduce(d, s, seq++, timeout, sh)))
                goto aborted;
            const double nlogG = sh.G, nlogH = sh.H;   // the refresh's totals (sh.G/H are reused below)
            double gk_d = 0.0, gk_a = 0.0;
            if (genkin) {
                double ds = 0.0, as = 0.0;
                for (long long k = d.shard_row[s] + threadIdx.x; k < d.shard_row[s + 1]; k += blockDim.x) {
                    const double e = d.E[k];
                    ds += fabs(log(e / d.E_prev[k]));
                    as += fabs(log(e / d.L[k]));
                    d.E_prev[k] = e;
                }
                bool gbad = false;
                const Fx fa = fx_from_double(ds, gbad), fb = fx_from_double(as, gbad);
                if (!block_grid_reduce(d, s, seq++, timeout, sh, fa, fb, gbad)) goto aborted;
                gk_d = sh.G;
                gk_a = sh.H;
            }
            if (threadIdx.x == 0) {
                const double lp = p.prior == 1 ? -0.5 * sh.sq * p.inv_var : (p.prior == 2 ? -p.lambda * sh.ab : 0.0);
                loglik = sh.lin - (nlogG - nlogH);
                P = loglik + lp;
                if (leader && p.record_history) hist[c] = P;
                conv = fabs(P - P_prev);
                if (p.tol_mode == 1) conv /= fmax(1.0, fabs(P));
                if (genkin) conv = gk_d / (1.0 + gk_a);
                cycles = c;
                if (!(P == P) || isinf(P)) status = kStNumeric;
                else if (status == kStNotConverged && p.tol >= 0.0 && conv < p.tol) status = kStOk;
                P_prev = P;
                sh.stop = status;
            }
            __syncthreads();
            status = sh.stop;
        }
        nonzero = sh.nonzero;
        if (threadIdx.x == 0) nonzero += nonzero_nar;
    }
    if (!F32 && p.ho_nev && (status == kStOk || status == kStNotConverged)) {
        // Section 2.5: the held-out fold's predictive log-likelihood at the final beta, from the
        // same state and with the same arithmetic as a separate evaluation (refresh, exact sums)
        DevLayout dh = d;
        dh.nev = p.ho_nev;
        dh.ytx = p.ho_ytx;
        if (!refresh_and_reduce(dh, s, seq++, timeout, sh)) goto aborted;
        if (threadIdx.x == 0) {
            double lin_ho = 0.0, lp_unused = 0.0;
            beta_terms(dh, s, p, lin_ho, lp_unused);
            heldout = lin_ho - (sh.G - sh.H);
        }
    }
    drain_stages(sh, pending, phase_bits, timeout);
    if (leader) {
        out->logpost = P;
        out->loglik = loglik;
        out->heldout_loglik = heldout;
        out->conv = conv;
        out->cycles = cycles;
        out->status = status;
        out->nonzero_steps = nonzero;
        out->warnings = warn;
        out->seq_end = seq;
        out->err_where = 0;
    }
    finish_run(sh, status, seq);
    return;
aborted:
    drain_stages(sh, pending, phase_bits, timeout);
    if (leader) {
        out->status = kStTimeout;
        out->err_where = 1;
    }
    finish_run(sh, kStTimeout, seq);
}


template <bool F32>
__global__ void __launch_bounds__(512, 1) fit_kernel(DevLayout d, FitParams p, FitOut *out, double *hist) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ SharedState sh;
    const bool clustered = p.cluster != 0;
    if (clustered) {
        // The cluster columns take CTA c of the first cluster as cluster shard c and address their
        // peers by cluster rank, so the launch must be in clusters of exactly C consecutive CTAs.
        // A CTA that finds otherwise (a launch that dropped the cluster shape) takes no step: it
        // sets the abort flag, every other CTA's waits give up, and the host reports the fit failed.
        unsigned cid, crank, csize;
        asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(cid));
        asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(crank));
        asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(csize));
        const bool shape_ok = csize == static_cast<unsigned>(d.C) && cid * csize + crank == blockIdx.x;
        // the cluster all-reduce's mbarriers (one arrival and C x 16 bytes a round) are initialised
        // in every CTA before any CTA of the cluster can send bytes to them
        if (threadIdx.x == 0) {
            mbar_init(&sh.cbar[0], 1);
            mbar_init(&sh.cbar[1], 1);
            mbar_init_fence();
            if (!shape_ok) {
                atomicExch(d.abort_flag, 1);
                out->err_where = 4;
            }
        }
        cluster_barrier_all();
        if (!shape_ok) {
            cluster_barrier_all();
            return;
        }
    }
    run_fit<F32>(d, p, out, hist, blockIdx.x, *reinterpret_cast<SmemLayout *>(smem_raw), sh);
    if (clustered) cluster_barrier_all();   // no CTA exits while another may still write its shared memory
}

// E_k = l_k exp(Xb_k) on shard s's rows, with Xb_k summed over row k's columns in ascending j;
// the shard's private beta copy = beta0 (0 when null) and its trust radii = 1 unless kept.
// beta0 may be the shard's own copy (a warm start).
// The same without the row index: column by column in j order, a block barrier after each.
__device__ void init_shard_by_columns(const DevLayout &d, int s, const double *beta0, bool keep_trust) {
    const long long r0 = d.shard_row[s], r1 = d.shard_row[s + 1];
    double *beta = d.beta_priv + static_cast<long long>(s) * d.J;
    double *trust = d.trust_priv + static_cast<long long>(s) * d.J;
    if (!beta0) {
        for (int j = threadIdx.x; j < d.J; j += blockDim.x) {
            beta[j] = 0.0;
            if (!keep_trust) trust[j] = 1.0;
        }
        for (long long k = r0 + threadIdx.x; k < r1; k += blockDim.x) d.E[k] = d.L[k];
        __syncthreads();
        return;
    }
    for (int j = threadIdx.x; j < d.J; j += blockDim.x) {
        beta[j] = beta0[j];
        if (!keep_trust) trust[j] = 1.0;
    }
    for (long long k = r0 + threadIdx.x; k < r1; k += blockDim.x) d.E[k] = 0.0;
    __syncthreads();
    for (int j = 0; j < d.J; ++j) {
        const double bj = beta0[j];
        if (bj == 0.0) continue;
        const long long so = static_cast<long long>(s) * (d.J + 1) + j;
        for (long long q = d.slice_row[so] + threadIdx.x; q < d.slice_row[so + 1]; q += blockDim.x)
            d.E[d.rows[q]] += bj;
        __syncthreads();
    }
    for (long long k = r0 + threadIdx.x; k < r1; k += blockDim.x) d.E[k] = d.L[k] * exp(d.E[k]);
    __syncthreads();
}

__device__ void init_shard(const DevLayout &d, int s, const double *beta0, bool keep_trust) {
    if (beta0 && d.row_ptr) {
        const long long r0 = d.shard_row[s], r1 = d.shard_row[s + 1];
        double *beta = d.beta_priv + static_cast<long long>(s) * d.J;
        double *trust = d.trust_priv + static_cast<long long>(s) * d.J;
        for (long long k = r0 + threadIdx.x; k < r1; k += blockDim.x) {
            double xb = 0.0;
            for (long long e = d.row_ptr[k]; e < d.row_ptr[k + 1]; ++e) xb += beta0[d.row_col[e]];
            d.E[k] = d.L[k] * exp(xb);
        }
        __syncthreads();   // every thread has read beta0 (possibly this shard's own copy)
        for (int j = threadIdx.x; j < d.J; j += blockDim.x) {
            beta[j] = beta0[j];
            if (!keep_trust) trust[j] = 1.0;
        }
        __syncthreads();
        return;
    }
    init_shard_by_columns(d, s, beta0, keep_trust);
}

__device__ void e_to_f32_shard(const DevLayout &d, int s) {
    for (long long k = d.shard_row[s] + threadIdx.x; k < d.shard_row[s + 1]; k += blockDim.x)
        d.E32[k] = static_cast<float>(d.E[k]);
    __syncthreads();
}

// Wait until all `team` CTAs of a fit have arrived (bounded; gives up early if the fit was
// aborted).  Thread 0 only.
__device__ bool team_assemble(unsigned *arrived, int team, long long limit_ns, int *abort_flag) {
    __threadfence();
    atomicAdd(arrived, 1u);
    const long long t0 = now_ns();
    for (unsigned it = 0;; ++it) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(arrived) : "memory");
        if (static_cast<int>(v) >= team) return true;
        if (*reinterpret_cast<volatile int *>(abort_flag)) return false;
        if ((it & 63u) == 63u && now_ns() - t0 > limit_ns) {
            atomicExch(abort_flag, 1);
            return false;
        }
        __nanosleep(200);
    }
}

// Several independent fits in one persistent launch, scheduled as a ticket queue (one ticket
// per CTA of each fit's team, in the host's order).  A team's CTAs exchange partial sums only
// with each other, through the fit's own all-reduce slots, so teams never wait on one another
// and every fit computes exactly what it computes when launched alone with the same shards.
template <int MODE>
__global__ void __launch_bounds__(512, 1) fit_queue_kernel(const BatchEntry *entries, const int *team_start, int n,
                                                          unsigned *counters, long long assemble_ns) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ SharedState sh;
    __shared__ __align__(16) BatchEntry e;
    __shared__ int sh_t, sh_f, sh_go;
    SmemLayout &sm = *reinterpret_cast<SmemLayout *>(smem_raw);
    const int total = team_start[n];
    if (threadIdx.x == 0) sh.drained = 1;
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = static_cast<int>(atomicAdd(&counters[0], 1u));
            int f = -1;
            if (t < total) {
                int lo = 0, hi = n - 1;             // largest f with team_start[f] <= t
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (team_start[mid] <= t) lo = mid;
                    else hi = mid - 1;
                }
                f = lo;
            }
            sh_t = t;
            sh_f = f;
        }
        __syncthreads();
        const int t = sh_t, f = sh_f;
        if (t >= total) break;
        {
            const int *src = reinterpret_cast<const int *>(entries + f);
            int *dst = reinterpret_cast<int *>(&e);
            for (int i = threadIdx.x; i < static_cast<int>(sizeof(BatchEntry) / sizeof(int)); i += blockDim.x)
                dst[i] = src[i];
        }
        __syncthreads();
        const int s = t - team_start[f];
        init_shard(e.d, s, e.warm ? e.d.beta_priv + static_cast<long long>(s) * e.d.J : nullptr, false);
        if (MODE != kBatchFp64) e_to_f32_shard(e.d, s);
        if (threadIdx.x == 0) sh_go = team_assemble(&counters[1 + f], e.team, assemble_ns, e.d.abort_flag) ? 1 : 0;
        __syncthreads();
        if (!sh_go) {
            if (threadIdx.x == 0 && s == 0) {
                e.out->status = kStTimeout;
                e.out->err_where = 3;
            }
            __syncthreads();
            continue;
        }
        if (MODE == kBatchFp64) {
            run_fit<false>(e.d, e.p, e.out, e.hist, s, sm, sh);
        } else if (MODE == kBatchFp32) {
            run_fit<true>(e.d, e.p32, e.out, e.hist, s, sm, sh);
        } else {
            run_fit<true>(e.d, e.p32, e.out32, e.hist, s, sm, sh);
            const int st = sh.run_status;
            if ((st == kStOk || st == kStNotConverged) && sh.drained) {
                // FP64 polish from the FP32 point: E and D rebuilt in FP64 from this shard's
                // copy of beta (every shard holds the same one), trust radii kept
                init_shard(e.d, s, e.d.beta_priv + static_cast<long long>(s) * e.d.J, true);
                FitParams p2 = e.p;
                p2.seq0 = sh.run_seq;
                run_fit<false>(e.d, p2, e.out, e.hist, s, sm, sh);
            }
        }
        if (!sh.drained) break;   // a staging copy may still land: this CTA takes no more work
    }
}

__global__ void batch_prep_kernel(const BatchEntry *entries, int n, unsigned *counters) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x) {
        counters[i] = 0u;
        if (i < n) {
            FitOut z{};
            *entries[i].out = z;
            if (entries[i].out32) *entries[i].out32 = z;
        }
    }
}

__global__ void batch_gather_kernel(const BatchEntry *entries, int n, FitOut *outs, FitOut *outs32, double *betas,
                                    const long long *beta_off) {
    for (int f = blockIdx.x; f < n; f += gridDim.x) {
        const BatchEntry &en = entries[f];
        if (threadIdx.x == 0) {
            outs[f] = *en.out;
            if (en.out32) outs32[f] = *en.out32;
        }
        for (int j = threadIdx.x; j < en.d.J; j += blockDim.x) betas[beta_off[f] + j] = en.d.beta_priv[j];
    }
}

__global__ void __launch_bounds__(512, 1) grad_hess_kernel(DevLayout d, int j, FitParams p, FitOut *out) {
    __shared__ SharedState sh;
    const long long timeout = p.timeout_ns;
    unsigned long long seq = p.seq0;
    if (!refresh_and_reduce(d, blockIdx.x, seq++, timeout, sh)) goto aborted;
    {
        double G = 0.0, H = 0.0;
        bool bad = false;
        phase_a_global<false>(d, blockIdx.x, j, nullptr, G, H, bad);
        const Fx fg = fx_from_double(G, bad), fh = fx_from_double(H, bad);
        if (!block_grid_reduce(d, blockIdx.x, seq++, timeout, sh, fg, fh, bad)) goto aborted;
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

__global__ void __launch_bounds__(512, 1) init_state_kernel(DevLayout d, const double *beta0, int keep_trust) {
    init_shard(d, blockIdx.x, beta0, keep_trust != 0);
}

__global__ void __launch_bounds__(512, 1) e_to_f32_kernel(DevLayout d) { e_to_f32_shard(d, blockIdx.x); }

// Section 2.5 weights: w_i n_i per subject (grid-stride) and, one block per column, the
// weighted Y'X_j as an exact integer sum over the column's (subject, y) pairs.
__global__ void __launch_bounds__(256) weighted_counts_kernel(DevLayout d, const int32_t *w, int32_t *nev_w,
                                                              double *ytx_w) {
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < d.N;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        nev_w[i] = w[i] * d.nev[i];
    __shared__ long long part[8];
    for (int j = blockIdx.x; j < d.J; j += gridDim.x) {
        long long t = 0;
        for (long long e = d.ycol_ptr[j] + threadIdx.x; e < d.ycol_ptr[j + 1]; e += blockDim.x)
            t += static_cast<long long>(w[d.ysub[e]]) * d.ycnt[e];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = t;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long s = 0;
            for (int q = 0; q < static_cast<int>(blockDim.x >> 5); ++q) s += part[q];
            ytx_w[j] = static_cast<double>(s);
        }
        __syncthreads();
    }
}

// ---- row -> columns index (for rebuilding E from a beta without a barrier per column)

constexpr int kScanChunk = 8192;   // rows per block of the prefix sum

// Each (shard, column) slice adds one to the count of every row it holds.
__global__ void __launch_bounds__(256) row_count_kernel(DevLayout d, int32_t *cnt) {
    const long long slices = static_cast<long long>(d.S) * d.J;
    for (long long t = blockIdx.x; t < slices; t += gridDim.x) {
        const int s = static_cast<int>(t / d.J), j = static_cast<int>(t % d.J);
        const long long so = static_cast<long long>(s) * (d.J + 1) + j;
        for (long long q = d.slice_row[so] + threadIdx.x; q < d.slice_row[so + 1]; q += blockDim.x)
            atomicAdd(&cnt[d.rows[q]], 1);
    }
}

__device__ long long block_sum_ll(long long v, long long *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    long long t = 0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += red[w];
    return t;
}

// Prefix sum, pass 1: the total of each chunk of kScanChunk counts.
__global__ void __launch_bounds__(256) scan_chunk_sums_kernel(const int32_t *cnt, long long n, long long *sums) {
    __shared__ long long red[8];
    const long long a = static_cast<long long>(blockIdx.x) * kScanChunk;
    const long long b = a + kScanChunk < n ? a + kScanChunk : n;
    long long v = 0;
    for (long long i = a + threadIdx.x; i < b; i += blockDim.x) v += cnt[i];
    const long long t = block_sum_ll(v, red);
    if (threadIdx.x == 0) sums[blockIdx.x] = t;
}

// Pass 2 (one thread): exclusive prefix of the chunk totals.
__global__ void scan_chunk_offsets_kernel(long long *sums, long long nchunks) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    long long run = 0;
    for (long long c = 0; c < nchunks; ++c) {
        const long long v = sums[c];
        sums[c] = run;
        run += v;
    }
    sums[nchunks] = run;
}

// Pass 3: each chunk's exclusive prefix, one warp-serial run per 32-count stretch; also the
// fill cursors (a copy of the offsets).
__global__ void __launch_bounds__(256) scan_chunk_fill_kernel(const int32_t *cnt, long long n, const long long *sums,
                                                              int64_t *row_ptr, int64_t *cursor) {
    __shared__ long long part[256];
    const long long a = static_cast<long long>(blockIdx.x) * kScanChunk;
    const long long b = a + kScanChunk < n ? a + kScanChunk : n;
    constexpr int per = kScanChunk / 256;
    const long long lo = a + static_cast<long long>(threadIdx.x) * per;
    long long v = 0;
    for (long long i = lo; i < lo + per && i < b; ++i) v += cnt[i];
    part[threadIdx.x] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long run = sums[blockIdx.x];
        for (int t = 0; t < 256; ++t) {
            const long long x = part[t];
            part[t] = run;
            run += x;
        }
    }
    __syncthreads();
    long long run = part[threadIdx.x];
    for (long long i = lo; i < lo + per && i < b; ++i) {
        row_ptr[i] = run;
        cursor[i] = run;
        run += cnt[i];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) row_ptr[n] = sums[gridDim.x];
}

// Scatter column ids into their rows (order within a row not yet fixed).
__global__ void __launch_bounds__(256) row_fill_kernel(DevLayout d, int64_t *cursor, int32_t *row_col) {
    const long long slices = static_cast<long long>(d.S) * d.J;
    for (long long t = blockIdx.x; t < slices; t += gridDim.x) {
        const int s = static_cast<int>(t / d.J), j = static_cast<int>(t % d.J);
        const long long so = static_cast<long long>(s) * (d.J + 1) + j;
        for (long long q = d.slice_row[so] + threadIdx.x; q < d.slice_row[so + 1]; q += blockDim.x) {
            const long long at = static_cast<long long>(atomicAdd(reinterpret_cast<unsigned long long *>(&cursor[d.rows[q]]), 1ull));
            row_col[at] = j;
        }
    }
}

// Each row's columns ascending (insertion sort; rows hold a handful of columns).
__global__ void __launch_bounds__(256) row_sort_kernel(const int64_t *row_ptr, int32_t *row_col, long long K) {
    for (long long k = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; k < K;
         k += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long a = row_ptr[k], b = row_ptr[k + 1];
        for (long long i = a + 1; i < b; ++i) {
            const int32_t v = row_col[i];
            long long m = i - 1;
            while (m >= a && row_col[m] > v) {
                row_col[m + 1] = row_col[m];
                --m;
            }
            row_col[m + 1] = v;
        }
    }
}

// Diagnostic: the step's e^x against CUDA's exp, element by element.
__global__ void exp_selftest_kernel(const double *x, long long n, double *ours, double *ref) {
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        ours[i] = exp_step(x[i]).r;
        ref[i] = exp(x[i]);
    }
}

// Diagnostic: the coordinate path's quotient against the IEEE division, element by element.
__global__ void div_selftest_kernel(const double *a, const double *b, long long n, double *ours, double *ref) {
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        ours[i] = quot(a[i], b[i]);
        ref[i] = a[i] / b[i];
    }
}

int ensure_smem_attr() {
    const int bytes = static_cast<int>(sizeof(SmemLayout));
    cudaError_t e = cudaFuncSetAttribute(fit_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fit_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)   // clusters of 16 CTAs are past the portable size of 8
        e = cudaFuncSetAttribute(fit_kernel<false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fit_queue_kernel<kBatchFp64>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fit_queue_kernel<kBatchFp32Polish>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fit_queue_kernel<kBatchFp32>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return static_cast<int>(e);
}

}  // namespace

size_t fit_kernel_smem_bytes() { return sizeof(SmemLayout); }

int launch_init_state(const DevLayout &d, const double *beta0_dev, int threads, void *stream, bool keep_trust) {
    init_state_kernel<<<d.S, threads, 0, static_cast<cudaStream_t>(stream)>>>(d, beta0_dev, keep_trust ? 1 : 0);
    return static_cast<int>(cudaGetLastError());
}

int launch_e_to_f32(const DevLayout &d, int threads, void *stream) {
    e_to_f32_kernel<<<d.S, threads, 0, static_cast<cudaStream_t>(stream)>>>(d);
    return static_cast<int>(cudaGetLastError());
}

int launch_exp_selftest(const double *x, long long n, double *ours, double *ref, void *stream) {
    const int blocks = static_cast<int>(std::min<long long>(std::max<long long>((n + 255) / 256, 1), 1024));
    exp_selftest_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(x, n, ours, ref);
    return static_cast<int>(cudaGetLastError());
}

int launch_div_selftest(const double *a, const double *b, long long n, double *ours, double *ref, void *stream) {
    const int blocks = static_cast<int>(std::min<long long>(std::max<long long>((n + 255) / 256, 1), 1024));
    div_selftest_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(a, b, n, ours, ref);
    return static_cast<int>(cudaGetLastError());
}

size_t row_index_scan_blocks(int64_t K) { return static_cast<size_t>((K + kScanChunk - 1) / kScanChunk) + 2; }

int launch_build_row_index(const DevLayout &d, int64_t *row_ptr, int32_t *row_col, int32_t *cnt, int64_t *cursor,
                           int64_t *block_sums, void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long K = d.K;
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * static_cast<size_t>(K > 0 ? K : 1), st);
    if (e != cudaSuccess) return static_cast<int>(e);
    const long long slices = static_cast<long long>(d.S) * d.J;
    const int sgrid = static_cast<int>(std::min<long long>(std::max<long long>(slices, 1), 65536));
    if (slices > 0) row_count_kernel<<<sgrid, 256, 0, st>>>(d, cnt);
    const long long nchunks = (K + kScanChunk - 1) / kScanChunk;
    long long *sums = reinterpret_cast<long long *>(block_sums);
    if (nchunks > 0) {
        scan_chunk_sums_kernel<<<static_cast<unsigned>(nchunks), 256, 0, st>>>(cnt, K, sums);
        scan_chunk_offsets_kernel<<<1, 32, 0, st>>>(sums, nchunks);
        scan_chunk_fill_kernel<<<static_cast<unsigned>(nchunks), 256, 0, st>>>(cnt, K, sums, row_ptr, cursor);
    } else {
        e = cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), st);
        if (e != cudaSuccess) return static_cast<int>(e);
    }
    if (slices > 0) row_fill_kernel<<<sgrid, 256, 0, st>>>(d, cursor, row_col);
    if (K > 0) {
        const int kgrid = static_cast<int>(std::min<long long>((K + 255) / 256, 65536));
        row_sort_kernel<<<kgrid, 256, 0, st>>>(row_ptr, row_col, K);
    }
    return static_cast<int>(cudaGetLastError());
}

int launch_weighted_counts(const DevLayout &d, const int32_t *w_kept, int32_t *nev_w, double *ytx_w, void *stream) {
    // a modest grid: the kernel is short, and fits running beside it need whole SMs
    const long long want = std::max<long long>(static_cast<long long>(d.J), (d.N + 255) / 256);
    const int blocks = static_cast<int>(std::min<long long>(std::max<long long>(want, 1), std::max(2 * d.S, 16)));
    weighted_counts_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(d, w_kept, nev_w, ytx_w);
    return static_cast<int>(cudaGetLastError());
}

int launch_fit(const DevLayout &d, const FitParams &p, FitOut *out_dev, double *hist_dev, int threads,
               void *stream, bool fp32) {
    int e = ensure_smem_attr();
    if (e) return e;
    DevLayout dd = d;
    FitParams pp = p;
    // FP64 fits of a layout with cluster columns launch in clusters of d.C CTAs
    pp.cluster = (!fp32 && d.C > 0 && d.S % d.C == 0) ? 1 : 0;
    // Phase C of a slice too big to stage takes E from the stash phase A wrote.  Gathering it
    // again instead moves less DRAM (9.44 against 10.66 GB per launch on the 1M-subject fit, whose
    // E fits the L2) but was 0.65% slower there (27.13 against 26.95 ms, same box, twice), and
    // slower still where E does not fit the L2.
    pp.regather_e = (!fp32 && SCCS_REGATHER_E) ? 1 : 0;
    void *args[] = {&dd, &pp, &out_dev, &hist_dev};
    void *fn = fp32 ? reinterpret_cast<void *>(fit_kernel<true>) : reinterpret_cast<void *>(fit_kernel<false>);
    if (!pp.cluster)
        return static_cast<int>(cudaLaunchCooperativeKernel(fn, dim3(d.S), dim3(threads), args, sizeof(SmemLayout),
                                                             static_cast<cudaStream_t>(stream)));
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(d.S);
    cfg.blockDim = dim3(threads);
    // a cluster launch runs no narrow columns, so the layout's last member (the second narrow
    // buffer) is left out: 57 KB more of the SM's unified memory stays L1 cache (1% faster, A/B)
    cfg.dynamicSmemBytes = sizeof(SmemLayout) - sizeof(NarrowBuf);
    cfg.stream = static_cast<cudaStream_t>(stream);
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = static_cast<unsigned>(d.C);
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return static_cast<int>(cudaLaunchKernelExC(&cfg, fn, args));
}

int fit_kernel_max_clusters(int threads, int cluster, int *clusters) {
    *clusters = 0;
    int e = ensure_smem_attr();
    if (e) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(static_cast<unsigned>(cluster));
    cfg.blockDim = dim3(static_cast<unsigned>(threads));
    cfg.dynamicSmemBytes = sizeof(SmemLayout);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = static_cast<unsigned>(cluster);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t ce = cudaOccupancyMaxActiveClusters(clusters, reinterpret_cast<const void *>(fit_kernel<false>), &cfg);
    if (ce != cudaSuccess) {
        (void)cudaGetLastError();
        *clusters = 0;
        return static_cast<int>(ce);
    }
    return 0;
}

int launch_fit_queue(const BatchEntry *entries_dev, const int *team_start_dev, int n, unsigned *counters_dev,
                     int ctas, int threads, void *stream, int mode, long long assemble_ns) {
    int e = ensure_smem_attr();
    if (e) return e;
    const BatchEntry *en = entries_dev;
    const int *ts = team_start_dev;
    int nn = n;
    unsigned *cn = counters_dev;
    long long an = assemble_ns;
    void *args[] = {&en, &ts, &nn, &cn, &an};
    void *fn = mode == kBatchFp32Polish ? reinterpret_cast<void *>(fit_queue_kernel<kBatchFp32Polish>)
               : mode == kBatchFp32     ? reinterpret_cast<void *>(fit_queue_kernel<kBatchFp32>)
                                        : reinterpret_cast<void *>(fit_queue_kernel<kBatchFp64>);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = sizeof(SmemLayout);
    cfg.stream = static_cast<cudaStream_t>(stream);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return static_cast<int>(cudaLaunchKernelExC(&cfg, fn, args));
}

int launch_batch_prep(const BatchEntry *entries_dev, int n, unsigned *counters_dev, void *stream) {
    const int blocks = (n + 1 + 255) / 256;
    batch_prep_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(entries_dev, n, counters_dev);
    return static_cast<int>(cudaGetLastError());
}

int launch_batch_gather(const BatchEntry *entries_dev, int n, FitOut *outs, FitOut *outs32, double *betas,
                        const long long *beta_off_dev, void *stream) {
    const int blocks = n < 1024 ? n : 1024;
    batch_gather_kernel<<<blocks, 128, 0, static_cast<cudaStream_t>(stream)>>>(entries_dev, n, outs, outs32, betas,
                                                                              beta_off_dev);
    return static_cast<int>(cudaGetLastError());
}

int launch_grad_hess(const DevLayout &d, int32_t j, const FitParams &p, FitOut *out_dev, int threads,
                     void *stream) {
    return launch_grad_hess_partial(d, j, p, out_dev, threads, d.S, stream);
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
    int e = ensure_smem_attr();
    if (e) return e;
    int a = 0, b = 0;
    cudaError_t ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, fit_kernel<false>, threads, sizeof(SmemLayout));
    if (ce != cudaSuccess) return static_cast<int>(ce);
    int c = 0;
    for (int m = 0; m < 3; ++m) {
        const void *fn = m == 0 ? reinterpret_cast<const void *>(fit_queue_kernel<kBatchFp64>)
                         : m == 1 ? reinterpret_cast<const void *>(fit_queue_kernel<kBatchFp32Polish>)
                                  : reinterpret_cast<const void *>(fit_queue_kernel<kBatchFp32>);
        ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, fn, threads, sizeof(SmemLayout));
        if (ce != cudaSuccess) return static_cast<int>(ce);
        if (c < a) a = c;
    }
    ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, grad_hess_kernel, threads, 0);
    if (ce != cudaSuccess) return static_cast<int>(ce);
    *blocks = a < b ? a : b;
    return 0;
}

}  // namespace sccs

// ====================================================================================
// Gradient and Hessian of one column with no device allocation.
//
// Some callers cannot allocate device memory at the point where they need this step: a
// serving process whose framework reserved all device memory up front for its own pool (a
// cudaMalloc there fails, or synchronises the device and stalls the other streams), or code
// called back from another library that forbids allocation.  For them the cross-CTA
// scratch of this reduction lives in a fixed array compiled into the library instead of a
// buffer from cudaMalloc.  Every device that loads the library holds the array until the
// process exits.
// ====================================================================================
namespace sccs {
namespace {

constexpr int kNoallocThreads = 256;
constexpr int kNoallocMaxBlocks = 4096;
// word 0: arrival counter; then 6 words (two exact sums) per CTA
constexpr int kNoallocWords = 8 + 6 * kNoallocMaxBlocks;

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoallocWords];

// One thread per segment: num = sum of E over the segment's rows, W = num / D, and the two
// exact partial sums; the last CTA to arrive adds every CTA's partial and writes g, h.
__global__ void __launch_bounds__(kNoallocThreads) grad_hess_noalloc_kernel(
    const int64_t *seg_ptr, const int32_t *seg_subject, const int32_t *rows, const double *E, const double *D,
    const int32_t *nev, double ytx, long long P, double *gh_out, unsigned long long *scratch) {
    __shared__ Fx wa[kNoallocThreads / 32], wb[kNoallocThreads / 32];
    __shared__ int wbad[kNoallocThreads / 32];
    __shared__ int is_last;
    const long long sidx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    bool bad = false;
    double gl = 0.0, hl = 0.0;
    if (sidx < P) {
        double num = 0.0;
        for (long long q = seg_ptr[sidx]; q < seg_ptr[sidx + 1]; ++q) num += E[rows[q]];
        const int i = seg_subject[sidx];
        segment_terms(num, D[i], nev[i], gl, hl, bad);
    }
    Fx fa = fx_warp_sum(fx_from_double(gl, bad));
    Fx fb = fx_warp_sum(fx_from_double(hl, bad));
    const int anybad = __any_sync(kFull, bad);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        wa[warp] = fa;
        wb[warp] = fb;
        wbad[warp] = anybad;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        Fx ta = lane < nw ? wa[lane] : fx_zero();
        Fx tb = lane < nw ? wb[lane] : fx_zero();
        const int cb = __any_sync(kFull, lane < nw ? wbad[lane] : 0);
        ta = fx_warp_sum(ta);
        tb = fx_warp_sum(tb);
        if (lane == 0) {
            unsigned long long *slot = scratch + 8 + 6 * static_cast<long long>(blockIdx.x);
            slot[0] = ta.w0; slot[1] = ta.w1; slot[2] = ta.w2;
            slot[3] = tb.w0; slot[4] = tb.w1; slot[5] = cb ? ~0ull : tb.w2;
            __threadfence();
            const unsigned long long prev = atomicAdd(&scratch[0], 1ull);
            is_last = prev == gridDim.x - 1;
        }
    }
    __syncthreads();
    if (!is_last || warp != 0) return;
    __threadfence();
    Fx sa = fx_zero(), sb = fx_zero();
    bool flag = false;
    for (unsigned b = lane; b < gridDim.x; b += 32) {
        const volatile unsigned long long *slot = scratch + 8 + 6 * static_cast<long long>(b);
        const Fx pa{slot[0], slot[1], slot[2]};
        const Fx pb{slot[3], slot[4], slot[5]};
        if (pb.w2 == ~0ull) flag = true;
        sa = fx_add(sa, pa);
        sb = fx_add(sb, pb);
    }
    sa = fx_warp_sum(sa);
    sb = fx_warp_sum(sb);
    flag = __any_sync(kFull, flag);
    if (lane == 0) {
        const double G = fx_to_double(sa), H = fx_to_double(sb);
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        gh_out[0] = flag ? nan : ytx - G;
        gh_out[1] = flag ? nan : -H;
        scratch[0] = 0ull;   // ready for the next call
    }
}

}  // namespace
}  // namespace sccs

namespace {
std::mutex g_noalloc_mu;
// Per device: the array's device address and the id of the context it was looked up in.  A
// context torn down and made again (cudaDeviceReset, say) maps the array elsewhere, so the
// address is looked up again whenever the current context's id differs.
void *g_noalloc_addr[64] = {};
unsigned long long g_noalloc_ctx[64] = {};

// The current context's id (unique for the life of the process), 0 if none is current.  The
// driver's functions come through the runtime, so the library does not link libcuda itself.
typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);
unsigned long long current_ctx_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        cudaDriverEntryPointQueryResult q1{}, q2{};
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f2);
        (void)cudaGetLastError();
        looked_up = true;
    }
    if (!get_current || !get_id) return 0;
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}
}  // namespace

extern "C" int sccs_grad_hess_noalloc(const int64_t *seg_ptr, const int32_t *seg_subject, const int32_t *rows,
                                      const double *E, const double *D, const int32_t *n, double ytx,
                                      int64_t P, double *gh_out, void *stream) {
    if (P < 0 || P > SCCS_NOALLOC_MAX_SEGMENTS)
        return sccs_set_error(SCCS_E_INVAL, "P must be in [0, SCCS_NOALLOC_MAX_SEGMENTS] (1048576 segments)");
    if (!gh_out || (P > 0 && (!seg_ptr || !seg_subject || !rows || !E || !D || !n)))
        return sccs_set_error(SCCS_E_INVAL, "null device pointer");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return sccs_set_error(SCCS_E_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return sccs_set_error(SCCS_E_INVAL, "device ordinal above 63");
    void *scratch = nullptr;
    {
        // First call on a device (or in a new context on it): look up the device address of the
        // array with the device current.  Host code must not pass the array's name itself to a
        // kernel: on the host that name is a stand-in, not a device address.
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        const unsigned long long ctx = current_ctx_id();
        if (!g_noalloc_addr[dev] || ctx == 0 || ctx != g_noalloc_ctx[dev]) {
            void *addr = nullptr;
            e = cudaGetSymbolAddress(&addr, sccs::g_noalloc_scratch);   // makes the context current if needed
            if (e != cudaSuccess) {
                g_noalloc_addr[dev] = nullptr;
                g_noalloc_ctx[dev] = 0;
                return sccs_set_error(SCCS_E_CUDA, cudaGetErrorString(e));
            }
            g_noalloc_addr[dev] = addr;
            g_noalloc_ctx[dev] = current_ctx_id();
        }
        scratch = g_noalloc_addr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the arrival counter must start at zero; the rest is overwritten before it is read
    e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return sccs_set_error(SCCS_E_CUDA, cudaGetErrorString(e));
    const long long blocks = P > 0 ? (P + sccs::kNoallocThreads - 1) / sccs::kNoallocThreads : 1;
    sccs::grad_hess_noalloc_kernel<<<static_cast<unsigned>(blocks), sccs::kNoallocThreads, 0, st>>>(
        seg_ptr, seg_subject, rows, E, D, n, ytx, P, gh_out, static_cast<unsigned long long *>(scratch));
    e = cudaGetLastError();
    if (e != cudaSuccess) return sccs_set_error(SCCS_E_CUDA, cudaGetErrorString(e));
    return SCCS_OK;
}
