// Check of the narrow-column layout the library builds at sccs_create (fetched through the
// layout diagnostic): every group's columns touch pairwise disjoint
// subjects and fit half the shared buffers, and every segment's mark names exactly the one
// earlier step that can change its subject -- the wide column before the run (for a run's
// first group) or the column of the previous group holding the same subject -- checked by
// brute force over the columns.  Exit status 0 when all hold (2: the handle could not be made).
// Needs a GPU.  Test infrastructure only.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <random>
#include <set>

#include "../../paper_1208_0945_gb300/csrc/sccs_internal.h"
#include "layout_fetch.h"

int main(int argc, char **argv) {
    const int nsub = argc > 1 ? atoi(argv[1]) : 20000;
    const int J = argc > 2 ? atoi(argv[2]) : 400;
    const unsigned seed = argc > 3 ? static_cast<unsigned>(atoi(argv[3])) : 7u;
    const int S = argc > 4 ? atoi(argv[4]) : 8;
    const int group_max = argc > 5 ? atoi(argv[5]) : 8;
    std::mt19937_64 rng(seed);
    std::vector<int64_t> pid;
    std::vector<int32_t> y;
    std::vector<double> L;
    for (int i = 0; i < nsub; ++i) {            // every subject has an event: none is dropped
        const int k = 1 + static_cast<int>(rng() % 8);
        for (int t = 0; t < k; ++t) {
            pid.push_back(i);
            y.push_back(t == 0 ? 1 : static_cast<int>(rng() % 2));
            L.push_back(1.0 + static_cast<double>(rng() % 365));
        }
    }
    const int64_t K = static_cast<int64_t>(pid.size());
    std::vector<int64_t> cp(J + 1, 0);
    std::vector<int32_t> ri;
    for (int j = 0; j < J; ++j) {               // heavy-tailed sizes, every 17th column wide
        const double u = static_cast<double>(rng() % 1000000) / 1e6;
        int64_t n = static_cast<int64_t>(5.0 / std::pow(1.0 - 0.999 * u, 1.2));
        if (j % 17 == 0) n = K / 20;
        std::set<int32_t> rows;
        while (static_cast<int64_t>(rows.size()) < std::min<int64_t>(n, K)) rows.insert(static_cast<int32_t>(rng() % K));
        for (int32_t r : rows) ri.push_back(r);
        cp[j + 1] = static_cast<int64_t>(ri.size());
    }
    sccs_create_opts o{};
    o.struct_size = sizeof(o);
    o.num_shards = S;
    o.cluster_ctas = -1;
    o.narrow_max_nnz = 1024;
    o.narrow_group_max = group_max;
    sccs_handle *h = nullptr;
    if (sccs_create(&h, K, pid.data(), y.data(), L.data(), J, cp.data(), ri.data(), nullptr, &o) != SCCS_OK) {
        printf("sccs_create failed: %s\n", sccs_last_error(nullptr));
        return 2;
    }
    const Layout hl = load_layout(h);
    sccs_destroy(h);
    if (hl.N != nsub || hl.K != K) {
        printf("unexpected subject drop\n");
        return 2;
    }
    std::vector<int32_t> row_sub(static_cast<size_t>(K));
    for (int i = 0; i < nsub; ++i)
        for (int64_t k = hl.pat_ptr[i]; k < hl.pat_ptr[i + 1]; ++k) row_sub[k] = i;
    auto col_has = [&](int j, int i) {
        for (int64_t e = cp[j]; e < cp[j + 1]; ++e)
            if (row_sub[ri[e]] == i) return true;
        return false;
    };
    long long checked = 0, bad = 0, after_wide = 0, after_prev = 0, groups = 0, runs = 0, multi = 0;
    int prev_group = -1;
    for (int g = 0; g < J;) {
        if (!hl.narrow[g]) {
            ++g;
            prev_group = -1;
            continue;
        }
        const int m = hl.nar_group[g];
        const bool run_start = g == 0 || !hl.narrow[g - 1];
        if (m < 1 || m > group_max || m > sccs::kNarrowGroupMax) {
            printf("group at %d: bad size %d\n", g, m);
            return 1;
        }
        runs += run_start;
        ++groups;
        multi += m > 1;
        // disjoint subjects, half-buffer fit, group-relative rows contiguous
        std::set<int32_t> subj;
        int64_t segs = hl.nar_ptr[g + m] - hl.nar_ptr[g], rows = 0;
        for (int c = 0; c < m; ++c) {
            if (!hl.narrow[g + c] || (c > 0 && hl.nar_group[g + c] != 0)) {
                printf("group at %d: column %d is not a member\n", g, g + c);
                return 1;
            }
            for (int64_t q = hl.nar_ptr[g + c]; q < hl.nar_ptr[g + c + 1]; ++q) {
                if (!subj.insert(hl.nar_seg[q].x).second) {
                    printf("group at %d: subject %d in two columns\n", g, hl.nar_seg[q].x);
                    return 1;
                }
                rows += hl.nar_seg[q].y;
            }
        }
        if (segs > sccs::kSegCap / 2 || rows > sccs::kRowCap / 2) {
            printf("group at %d: %lld segments, %lld rows exceed half the buffers\n", g, (long long)segs, (long long)rows);
            return 1;
        }
        for (int c = 0; c < m; ++c)
            for (int64_t q = hl.nar_ptr[g + c]; q < hl.nar_ptr[g + c + 1]; ++q) {
                const int i = hl.nar_seg[q].x;
                int want = 0;
                if (run_start) {
                    if (g > 0 && col_has(g - 1, i)) want = sccs::kNarrowAfterWide;
                } else {
                    for (int pc = 0; pc < hl.nar_group[prev_group]; ++pc)
                        if (col_has(prev_group + pc, i)) {
                            want = pc + 1;
                            break;
                        }
                }
                ++checked;
                after_wide += want == sccs::kNarrowAfterWide;
                after_prev += want > 0 && want <= sccs::kNarrowGroupMax;
                if (hl.nar_seg[q].w != want) {
                    if (bad < 5) printf("column %d segment %lld subject %d: mark %d, want %d\n", g + c, (long long)q, i, hl.nar_seg[q].w, want);
                    ++bad;
                }
            }
        prev_group = g;
        g += m;
    }
    printf("narrow %d runs %lld groups %lld multi %lld segments %lld after_wide %lld after_prev %lld mismatches %lld\n",
           hl.narrow_count, runs, groups, multi, checked, after_wide, after_prev, bad);
    return bad != 0 ? 1 : 0;
}
