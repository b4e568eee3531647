// Check of the whole layout the library builds on the device at sccs_create (fetched through
// the layout diagnostic), against a brute-force construction from the definitions: the kept
// subjects (n_i > 0, input order) and their rows, each column's kept rows and Y'X_j, the
// per-column (subject, event sum) pairs, and every (shard, column) slice -- its rows, its subject
// segments longest first (ties in subject order), the rows of each 32-segment group diagonal by
// diagonal, the group bases -- and the stash strides.  The data has subjects without events and
// columns in shuffled order, or neither, so every path of the layout stages runs.  Exit status 0
// when all hold (2: the handle could not be made).  Needs a GPU.  Test infrastructure only.
#include <algorithm>
#include <cstdlib>
#include <cstdio>
#include <map>
#include <iterator>
#include <random>
#include <string>

#include "../../paper_1208_0945_gb300/csrc/sccs_internal.h"
#include "layout_fetch.h"

static long long g_bad = 0;
#define CHECK(cond, ...)                      \
    do {                                      \
        if (!(cond)) {                        \
            if (g_bad < 8) printf(__VA_ARGS__); \
            ++g_bad;                          \
        }                                     \
    } while (0)

int main(int argc, char **argv) {
    const int nsub = argc > 1 ? atoi(argv[1]) : 8000;
    const int J = argc > 2 ? atoi(argv[2]) : 120;
    const unsigned seed = argc > 3 ? static_cast<unsigned>(atoi(argv[3])) : 5u;
    const int S = argc > 4 ? atoi(argv[4]) : 7;
    const bool messy = argc > 5 ? atoi(argv[5]) != 0 : true;   // dropped subjects, shuffled columns
    const int C = argc > 6 ? atoi(argv[6]) : 0;                 // cluster partition (0: none)
    const int64_t cmax = argc > 7 ? atoll(argv[7]) : 0;         // cluster columns: at most this many nonzeros
    std::mt19937_64 rng(seed);
    std::vector<int64_t> pid;
    std::vector<int32_t> y;
    std::vector<double> L;
    for (int i = 0; i < nsub; ++i) {
        const int k = 1 + static_cast<int>(rng() % 14);
        const bool events = !messy || rng() % 4 != 0;
        for (int t = 0; t < k; ++t) {
            pid.push_back(3 * static_cast<int64_t>(i) + 1);          // ids need not be dense
            y.push_back(events ? (t == 0 ? 1 + static_cast<int>(rng() % 3) : static_cast<int>(rng() % 2)) : 0);
            L.push_back(1.0 + static_cast<double>(rng() % 365));
        }
    }
    const int64_t K = static_cast<int64_t>(pid.size());
    std::vector<int64_t> cp(J + 1, 0);
    std::vector<int32_t> ri;
    for (int j = 0; j < J; ++j) {
        int64_t n = j % 11 == 0 ? K / 4 : static_cast<int64_t>(rng() % 300);
        if (j % 29 == 5) n = 0;                                         // empty columns
        std::vector<char> used(static_cast<size_t>(K), 0);
        std::vector<int32_t> col;
        while (static_cast<int64_t>(col.size()) < n) {
            const int32_t r = static_cast<int32_t>(rng() % K);
            if (!used[r]) {
                used[r] = 1;
                col.push_back(r);
            }
        }
        if (messy) std::shuffle(col.begin(), col.end(), rng);
        else std::sort(col.begin(), col.end());
        for (int32_t r : col) ri.push_back(r);
        cp[j + 1] = static_cast<int64_t>(ri.size());
    }
    sccs_create_opts o{};
    o.struct_size = sizeof(o);
    o.num_shards = S;
    o.cluster_ctas = C > 0 ? C : -1;
    o.cluster_max_nnz = static_cast<int32_t>(std::min<int64_t>(cmax, 2000000000));
    sccs_handle *h = nullptr;
    if (sccs_create(&h, K, pid.data(), y.data(), L.data(), J, cp.data(), ri.data(), nullptr, &o) != SCCS_OK) {
        printf("sccs_create failed: %s\n", sccs_last_error(nullptr));
        return 2;
    }
    const Layout hl = load_layout(h);

    // ---- subjects and rows, from the definitions
    std::vector<int64_t> first;                      // input subjects' first rows
    for (int64_t k = 0; k < K; ++k)
        if (k == 0 || pid[k] != pid[k - 1]) first.push_back(k);
    first.push_back(K);
    const int64_t nin = static_cast<int64_t>(first.size()) - 1;
    std::vector<int64_t> kept_row(static_cast<size_t>(K), -1);   // input row -> kept row
    std::vector<int32_t> kept_sub;                               // kept row -> kept subject
    int64_t Nk = 0, Kk = 0;
    CHECK(hl.subjects_in == nin, "subjects_in %lld != %lld\n", (long long)hl.subjects_in, (long long)nin);
    for (int64_t i = 0; i < nin; ++i) {
        int64_t n = 0;
        for (int64_t k = first[i]; k < first[i + 1]; ++k) n += y[k];
        if (n == 0) continue;
        CHECK(hl.pat_ptr[Nk] == Kk, "pat_ptr[%lld]\n", (long long)Nk);
        CHECK(hl.nev[Nk] == n, "nev[%lld]\n", (long long)Nk);
        CHECK(hl.kept_from[Nk] == i, "kept_from[%lld]\n", (long long)Nk);
        for (int64_t k = first[i]; k < first[i + 1]; ++k) {
            CHECK(hl.L[Kk] == L[k], "L[%lld]\n", (long long)Kk);
            kept_row[k] = Kk++;
            kept_sub.push_back(static_cast<int32_t>(Nk));
        }
        ++Nk;
    }
    CHECK(hl.N == Nk && hl.K == Kk, "N/K %lld/%lld != %lld/%lld\n", (long long)hl.N, (long long)hl.K, (long long)Nk,
          (long long)Kk);
    CHECK(hl.pat_ptr[Nk] == Kk, "pat_ptr end\n");
    std::vector<int32_t> ykept(static_cast<size_t>(Kk));
    for (int64_t k = 0; k < K; ++k)
        if (kept_row[k] >= 0) ykept[kept_row[k]] = y[k];

    // ---- columns: kept rows ascending, Y'X_j, event pairs
    std::vector<std::vector<int32_t>> colrows(static_cast<size_t>(J));
    int64_t nnz = 0;
    for (int j = 0; j < J; ++j) {
        for (int64_t e = cp[j]; e < cp[j + 1]; ++e)
            if (kept_row[ri[e]] >= 0) colrows[j].push_back(static_cast<int32_t>(kept_row[ri[e]]));
        std::sort(colrows[j].begin(), colrows[j].end());
        nnz += static_cast<int64_t>(colrows[j].size());
        int64_t ytx = 0;
        std::map<int32_t, int32_t> pairs;
        for (int32_t r : colrows[j]) {
            ytx += ykept[r];
            if (ykept[r] > 0) pairs[kept_sub[r]] += ykept[r];
        }
        CHECK(hl.ytx[j] == static_cast<double>(ytx), "ytx[%d]\n", j);
        CHECK(hl.ycol_ptr[j + 1] - hl.ycol_ptr[j] == static_cast<int64_t>(pairs.size()), "pairs count col %d\n", j);
        int64_t q = hl.ycol_ptr[j];
        for (const auto &pr : pairs) {
            CHECK(hl.ysub[q] == pr.first && hl.ycnt[q] == pr.second, "pair col %d\n", j);
            ++q;
        }
    }
    CHECK(hl.nnz == nnz, "nnz\n");

    // ---- slices of one partition (S shards, or the C cluster shards) of the columns in_set
    auto check_slices = [&](const char *tag, int S_, const std::vector<int64_t> &shard_row, const std::vector<int64_t> &shard_pat,
                            const std::vector<int64_t> &slice_row, const std::vector<int64_t> &slice_seg,
                            const std::vector<int64_t> &slice_grp, const std::vector<int32_t> &hrows,
                            const std::vector<int2> &hsegs, const std::vector<int64_t> &hgrp, auto in_set,
                            int64_t &max_seg, int64_t &max_rows) {
        max_seg = 1;
        max_rows = 1;
        CHECK(shard_row[0] == 0 && shard_row[S_] == Kk && shard_pat[S_] == Nk, "%s shard ends\n", tag);
        for (int s = 0; s < S_; ++s) {
            const int64_t r0 = shard_row[s], r1 = shard_row[s + 1];
            CHECK(r0 == hl.pat_ptr[shard_pat[s]], "%s shard_row[%d]\n", tag, s);
            CHECK(r0 <= r1, "%s shard order %d\n", tag, s);
            for (int j = 0; j < J; ++j) {
                const int64_t idx = static_cast<int64_t>(s) * (J + 1) + j;
                std::vector<int32_t> rows;
                if (in_set(j))
                    for (int32_t r : colrows[j])
                        if (r >= r0 && r < r1) rows.push_back(r);
                // subjects in ascending order with their rows (ascending)
                std::vector<std::pair<int32_t, std::vector<int32_t>>> segs;
                for (int32_t r : rows) {
                    if (segs.empty() || segs.back().first != kept_sub[r]) segs.push_back({kept_sub[r], {}});
                    segs.back().second.push_back(r);
                }
                std::stable_sort(segs.begin(), segs.end(),
                                 [](const auto &a, const auto &b) { return a.second.size() > b.second.size(); });
                const int64_t nr = slice_row[idx + 1] - slice_row[idx];
                const int64_t ns = slice_seg[idx + 1] - slice_seg[idx];
                CHECK(nr == static_cast<int64_t>(rows.size()), "%s slice rows s%d j%d\n", tag, s, j);
                CHECK(ns == static_cast<int64_t>(segs.size()), "%s slice segs s%d j%d\n", tag, s, j);
                CHECK(slice_grp[idx + 1] - slice_grp[idx] == (ns + 31) / 32, "%s slice groups s%d j%d\n", tag, s, j);
                max_seg = std::max<int64_t>(max_seg, ns);
                max_rows = std::max<int64_t>(max_rows, nr);
                if (nr != static_cast<int64_t>(rows.size()) || ns != static_cast<int64_t>(segs.size())) continue;
                for (int64_t i = 0; i < ns; ++i) {
                    const int2 sg = hsegs[slice_seg[idx] + i];
                    CHECK(sg.x == segs[i].first && sg.y == static_cast<int>(segs[i].second.size()), "%s seg s%d j%d i%lld\n",
                          tag, s, j, (long long)i);
                }
                int64_t pos = slice_row[idx];
                for (int64_t g = 0; g * 32 < ns; ++g) {
                    CHECK(hgrp[slice_grp[idx] + g] == pos, "%s grp_base s%d j%d g%lld\n", tag, s, j, (long long)g);
                    const int64_t a = 32 * g, b = std::min<int64_t>(ns, a + 32);
                    const size_t maxlen = segs[a].second.size();
                    for (size_t t = 0; t < maxlen; ++t)
                        for (int64_t l = a; l < b; ++l)
                            if (segs[l].second.size() > t) {
                                CHECK(hrows[pos] == segs[l].second[t], "%s row s%d j%d pos%lld\n", tag, s, j, (long long)pos);
                                ++pos;
                            }
                }
            }
        }
    };
    int64_t max_seg = 1, max_rows = 1;
    check_slices("grid", S, hl.shard_row, hl.shard_pat, hl.slice_row, hl.slice_seg, hl.slice_grp, hl.rows, hl.segs,
                 hl.grp_base, [](int) { return true; }, max_seg, max_rows);
    // ---- cluster columns: every column with at most cmax nonzeros whose slices over the C cluster
    //      shards all fit the staging caps, their slices there, and the next-grid-column map
    int64_t ccount = 0;
    if (C > 0) {
        CHECK(hl.C == C, "cluster size\n");
        std::vector<int64_t> cpat(static_cast<size_t>(C) + 1), crow_b(static_cast<size_t>(C) + 1);
        for (int c = 0; c <= C; ++c) {
            cpat[c] = hl.cshard_pat[c];
            crow_b[c] = hl.cshard_row[c];
        }
        for (int j = 0; j < J; ++j) {
            bool want = static_cast<int64_t>(colrows[j].size()) <= cmax;
            for (int c = 0; want && c < C; ++c) {
                std::vector<int32_t> subs;
                int64_t nr = 0;
                for (int32_t r : colrows[j])
                    if (r >= crow_b[c] && r < crow_b[c + 1]) {
                        ++nr;
                        if (subs.empty() || subs.back() != kept_sub[r]) subs.push_back(kept_sub[r]);
                    }
                if (nr > sccs::kRowCap || static_cast<int64_t>(subs.size()) > sccs::kSegCap) want = false;
            }
            CHECK(hl.ccls[j] == (want ? 1 : 0), "cluster class of column %d\n", j);
            ccount += want ? 1 : 0;
        }
        CHECK(hl.cluster_count == ccount, "cluster count\n");
        int64_t cms = 1, cmr = 1;
        check_slices("cluster", C, crow_b, cpat, hl.cslice_row, hl.cslice_seg, hl.cslice_grp, hl.crows, hl.csegs,
                     hl.cgrp_base, [&](int j) { return hl.ccls[j] != 0; }, cms, cmr);
        // groups: greedy runs of consecutive cluster columns, pairwise disjoint in subjects, at most
        // gmax, whose slices on every cluster shard fit the staging caps together
        const int gmax = 8;
        auto subjects = [&](int j) {
            std::vector<int32_t> v;
            for (int32_t r : colrows[j]) v.push_back(kept_sub[r]);
            std::sort(v.begin(), v.end());
            v.erase(std::unique(v.begin(), v.end()), v.end());
            return v;
        };
        for (int j = 0; j < J;) {
            if (!hl.ccls[j]) {
                CHECK(hl.cgroup[j] == 0, "cgroup of grid column %d\n", j);
                ++j;
                continue;
            }
            std::vector<int32_t> used = subjects(j);
            std::vector<int64_t> rs(static_cast<size_t>(C), 0), ss(static_cast<size_t>(C), 0);
            auto add_counts = [&](int jj, std::vector<int64_t> &r_, std::vector<int64_t> &s_) {
                for (int c = 0; c < C; ++c) {
                    std::vector<int32_t> sb;
                    for (int32_t r : colrows[jj])
                        if (r >= crow_b[c] && r < crow_b[c + 1]) {
                            r_[c]++;
                            if (sb.empty() || sb.back() != kept_sub[r]) sb.push_back(kept_sub[r]);
                        }
                    s_[c] += static_cast<int64_t>(sb.size());
                }
            };
            add_counts(j, rs, ss);
            int m = 1;
            while (j + m < J && hl.ccls[j + m] && m < gmax) {
                std::vector<int32_t> sj = subjects(j + m), both;
                std::set_intersection(used.begin(), used.end(), sj.begin(), sj.end(), std::back_inserter(both));
                std::vector<int64_t> r2 = rs, s2 = ss;
                add_counts(j + m, r2, s2);
                bool fits = both.empty();
                for (int c = 0; c < C && fits; ++c) fits = r2[c] <= sccs::kRowCap && s2[c] <= sccs::kSegCap;
                if (!fits) break;
                std::vector<int32_t> u2;
                std::set_union(used.begin(), used.end(), sj.begin(), sj.end(), std::back_inserter(u2));
                used.swap(u2);
                rs.swap(r2);
                ss.swap(s2);
                ++m;
            }
            CHECK(hl.cgroup[j] == m, "cgroup at %d: %d != %d\n", j, hl.cgroup[j], m);
            for (int t = 1; t < m; ++t) CHECK(hl.cgroup[j + t] == 0, "cgroup inside a group at %d\n", j + t);
            j += m;
        }
    }
    if (C > 0) {
        int32_t first_grid = -1;
        for (int j = 0; j < J && first_grid < 0; ++j)
            if (!hl.ccls[j]) first_grid = j;
        CHECK(hl.first_grid == first_grid, "first grid column\n");
        for (int j = 0; j < J; ++j) {
            int32_t nx = -1;
            for (int t = 1; t <= J && nx < 0; ++t)
                if (!hl.ccls[(j + t) % J]) nx = (j + t) % J;
            CHECK(hl.next_grid[j] == nx, "next grid column after %d\n", j);
        }
    }
    CHECK(hl.stash_stride == max_seg && hl.estash_stride == max_rows, "stash strides\n");
    sccs_destroy(h);
    printf("subjects %lld kept %lld rows %lld nnz %lld shards %d columns %d cluster_columns %lld mismatches %lld\n",
           (long long)nin, (long long)Nk, (long long)Kk, (long long)nnz, S, J, (long long)ccount, g_bad);
    return g_bad ? 1 : 0;
}
