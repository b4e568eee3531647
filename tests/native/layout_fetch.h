// The data layout of a handle, copied to the host through the library's layout diagnostic
// (sccs_debug_layout), under the names the layout checks use.  Test infrastructure only.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <vector>

#include "sccs.h"

template <class T>
std::vector<T> fetch_layout(const sccs_handle *h, int which) {
    int64_t b = 0;
    if (sccs_debug_layout(h, which, nullptr, 0, &b) != SCCS_OK) {
        printf("sccs_debug_layout(%d) failed: %s\n", which, sccs_last_error(h));
        return {};
    }
    std::vector<T> v(static_cast<size_t>(b) / sizeof(T));
    if (b && sccs_debug_layout(h, which, v.data(), b, &b) != SCCS_OK)
        printf("sccs_debug_layout(%d) failed: %s\n", which, sccs_last_error(h));
    return v;
}

struct Layout {
    int64_t K = 0, N = 0, nnz = 0, subjects_in = 0, stash_stride = 0, estash_stride = 0;
    int32_t C = 0, narrow_count = 0, cluster_count = 0, first_grid = -1, first_wide = -1;
    std::vector<int64_t> pat_ptr, kept_from, slice_row, slice_seg, slice_grp, shard_row, shard_pat, grp_base, ycol_ptr,
        nar_ptr, cslice_row, cslice_seg, cslice_grp, cshard_row, cshard_pat, cgrp_base;
    std::vector<int32_t> nev, rows, ysub, ycnt, next_wide, nar_row, nar_group, next_grid, cgroup, crows;
    std::vector<int2> segs, csegs;
    std::vector<int4> nar_seg;
    std::vector<uint8_t> narrow, ccls;
    std::vector<double> L, ytx;
};

inline Layout load_layout(const sccs_handle *h) {
    Layout l;
    sccs_data_info info{};
    sccs_get_info(h, &info);
    l.K = info.rows_kept;
    l.N = info.subjects_kept;
    l.C = info.cluster_ctas;
    const std::vector<int64_t> sc = fetch_layout<int64_t>(h, SCCS_DBG_SCALARS);
    if (sc.size() >= 8) {
        l.nnz = sc[0];
        l.subjects_in = sc[1];
        l.narrow_count = static_cast<int32_t>(sc[2]);
        l.cluster_count = static_cast<int32_t>(sc[3]);
        l.first_grid = static_cast<int32_t>(sc[4]);
        l.stash_stride = sc[5];
        l.estash_stride = sc[6];
        l.first_wide = static_cast<int32_t>(sc[7]);
    }
    l.pat_ptr = fetch_layout<int64_t>(h, SCCS_DBG_PAT_PTR);
    l.kept_from = fetch_layout<int64_t>(h, SCCS_DBG_KEPT_FROM);
    l.nev = fetch_layout<int32_t>(h, SCCS_DBG_NEV);
    l.L = fetch_layout<double>(h, SCCS_DBG_L);
    l.ytx = fetch_layout<double>(h, SCCS_DBG_YTX);
    l.rows = fetch_layout<int32_t>(h, SCCS_DBG_ROWS);
    l.segs = fetch_layout<int2>(h, SCCS_DBG_SEGS);
    l.grp_base = fetch_layout<int64_t>(h, SCCS_DBG_GRP_BASE);
    l.slice_row = fetch_layout<int64_t>(h, SCCS_DBG_SLICE_ROW);
    l.slice_seg = fetch_layout<int64_t>(h, SCCS_DBG_SLICE_SEG);
    l.slice_grp = fetch_layout<int64_t>(h, SCCS_DBG_SLICE_GRP);
    l.shard_row = fetch_layout<int64_t>(h, SCCS_DBG_SHARD_ROW);
    l.shard_pat = fetch_layout<int64_t>(h, SCCS_DBG_SHARD_PAT);
    l.ycol_ptr = fetch_layout<int64_t>(h, SCCS_DBG_YCOL_PTR);
    l.ysub = fetch_layout<int32_t>(h, SCCS_DBG_YSUB);
    l.ycnt = fetch_layout<int32_t>(h, SCCS_DBG_YCNT);
    l.narrow = fetch_layout<uint8_t>(h, SCCS_DBG_NARROW);
    l.next_wide = fetch_layout<int32_t>(h, SCCS_DBG_NEXT_WIDE);
    l.nar_ptr = fetch_layout<int64_t>(h, SCCS_DBG_NAR_PTR);
    l.nar_seg = fetch_layout<int4>(h, SCCS_DBG_NAR_SEG);
    l.nar_row = fetch_layout<int32_t>(h, SCCS_DBG_NAR_ROW);
    l.nar_group = fetch_layout<int32_t>(h, SCCS_DBG_NAR_GROUP);
    l.ccls = fetch_layout<uint8_t>(h, SCCS_DBG_CCLS);
    l.next_grid = fetch_layout<int32_t>(h, SCCS_DBG_NEXT_GRID);
    l.cgroup = fetch_layout<int32_t>(h, SCCS_DBG_CGROUP);
    l.crows = fetch_layout<int32_t>(h, SCCS_DBG_CROWS);
    l.csegs = fetch_layout<int2>(h, SCCS_DBG_CSEGS);
    l.cgrp_base = fetch_layout<int64_t>(h, SCCS_DBG_CGRP_BASE);
    l.cslice_row = fetch_layout<int64_t>(h, SCCS_DBG_CSLICE_ROW);
    l.cslice_seg = fetch_layout<int64_t>(h, SCCS_DBG_CSLICE_SEG);
    l.cslice_grp = fetch_layout<int64_t>(h, SCCS_DBG_CSLICE_GRP);
    l.cshard_row = fetch_layout<int64_t>(h, SCCS_DBG_CSHARD_ROW);
    l.cshard_pat = fetch_layout<int64_t>(h, SCCS_DBG_CSHARD_PAT);
    return l;
}
