"""sccs_grad_hess_noalloc: the gradient/Hessian step for callers that cannot allocate device
memory where they call it (for example inside a serving process whose framework holds all
device memory in its own pool).  Its cross-CTA scratch is an array compiled into the library,
so this checks it against the handle-based sccs_grad_hess on the same inputs, twice in a row
(the second call reuses the array the first one left behind).  This file is collected last."""
import numpy as np
import pytest

from synth import make_dataset

pytestmark = pytest.mark.gpu


def column_segments(d, j):
    """Rows of column j grouped by subject (all subjects here have events, so none are dropped)."""
    rows = d.column(j).astype(np.int64)
    subj = d.patient_id[rows]
    starts = np.flatnonzero(np.r_[True, subj[1:] != subj[:-1]]) if rows.size else np.zeros(0, np.int64)
    seg_ptr = np.r_[starts, rows.size].astype(np.int64)
    return seg_ptr, subj[starts].astype(np.int32), rows.astype(np.int32)


def test_noalloc_matches_grad_hess_on_two_calls_in_a_row():
    import torch
    import paper_1208_0945_gb300 as P

    d = make_dataset(n_patients=40000, eras=("geometric", 6), J=8, columns=("density_range", 0.001, 0.3),
                     n_true=3, beta_sd=0.4, seed=4242)
    assert np.all(np.bincount(d.patient_id, weights=d.y) > 0)
    beta = np.random.default_rng(7).normal(0, 0.4, d.J)
    xb = np.zeros(d.K)
    for j in range(d.J):
        xb[d.column(j)] += beta[j]
    E = d.L * np.exp(xb)
    D = np.bincount(d.patient_id, weights=E)
    n = np.bincount(d.patient_id, weights=d.y).astype(np.int32)
    dev = torch.device("cuda", 0)
    tE = torch.tensor(E, device=dev)
    tD = torch.tensor(D, device=dev)
    tn = torch.tensor(n, device=dev)
    out = torch.zeros(2, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    with P.SCCSModel(d, device=0) as m:
        ref = [m.grad_hess(j, beta) for j in range(d.J)]
        for _ in range(2):
            for j in range(d.J):
                seg_ptr, seg_subj, rows = column_segments(d, j)
                t_ptr = torch.tensor(seg_ptr, device=dev)
                t_subj = torch.tensor(seg_subj, device=dev)
                t_rows = torch.tensor(rows if rows.size else np.zeros(1, np.int32), device=dev)
                ytx = float(d.y[rows].sum())
                P.sccs_grad_hess_noalloc(t_ptr.data_ptr(), t_subj.data_ptr(), t_rows.data_ptr(), tE.data_ptr(),
                                         tD.data_ptr(), tn.data_ptr(), ytx, seg_subj.size, out.data_ptr(), stream)
                torch.cuda.synchronize(dev)
                g, h = out.cpu().numpy()
                g_ref, h_ref = ref[j]
                assert abs(g - g_ref) <= 1e-12 * max(1.0, abs(g_ref)) + 1e-12 * abs(h_ref), (j, g, g_ref)
                assert abs(h - h_ref) <= 1e-12 * max(1.0, abs(h_ref)), (j, h, h_ref)


def test_noalloc_rejects_more_segments_than_its_scratch_holds():
    import paper_1208_0945_gb300 as P

    with pytest.raises(P.SCCSError) as ei:
        P.sccs_grad_hess_noalloc(1, 1, 1, 1, 1, 1, 0.0, P.sccs.NOALLOC_MAX_SEGMENTS + 1, 1, None)
    assert ei.value.code == -1 and "SCCS_NOALLOC_MAX_SEGMENTS" in str(ei.value)


def _call(P, t, ytx, nseg, out, stream):
    P.sccs_grad_hess_noalloc(t["seg_ptr"].data_ptr(), t["seg_subj"].data_ptr(), t["rows"].data_ptr(),
                             t["E"].data_ptr(), t["D"].data_ptr(), t["n"].data_ptr(), ytx, nseg, out.data_ptr(),
                             stream)


def test_noalloc_at_its_maximum_size_and_on_bad_inputs():
    """Every scratch slot in use (SCCS_NOALLOC_MAX_SEGMENTS one-row segments, one per subject),
    against the exact sum of the per-subject terms in float64, on two calls in a row; then a
    subject with D = 0 and an infinite E, which must give NaN for both g and h; then P = 0."""
    import math

    import torch
    import paper_1208_0945_gb300 as P

    nseg = P.sccs.NOALLOC_MAX_SEGMENTS
    rng = np.random.default_rng(11)
    E = rng.uniform(1.0, 365.0, 2 * nseg) * np.exp(rng.normal(0, 0.5, 2 * nseg))
    D = E[0::2] + E[1::2]                      # subject i: rows 2i (in the column) and 2i + 1
    n = rng.integers(1, 6, nseg).astype(np.int32)
    w = E[0::2] / D
    G = math.fsum(n * w)
    H = math.fsum(n * w * (1.0 - w))
    ytx = float(rng.integers(0, 3 * nseg))
    dev = torch.device("cuda", 0)
    t = {"seg_ptr": torch.arange(nseg + 1, dtype=torch.int64, device=dev),
         "seg_subj": torch.arange(nseg, dtype=torch.int32, device=dev),
         "rows": torch.arange(0, 2 * nseg, 2, dtype=torch.int32, device=dev),
         "E": torch.tensor(E, device=dev), "D": torch.tensor(D, device=dev), "n": torch.tensor(n, device=dev)}
    out = torch.zeros(2, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    for _ in range(2):
        out.fill_(-1.0)
        _call(P, t, ytx, nseg, out, stream)
        torch.cuda.synchronize(dev)
        g, h = out.cpu().numpy()
        assert abs(g - (ytx - G)) <= 1e-12 * max(1.0, abs(G)), (g, ytx - G)
        assert abs(h + H) <= 1e-12 * H, (h, -H)
    # a subject with D = 0, then an infinite E: NaN for both outputs
    t["D"][12345] = 0.0
    _call(P, t, ytx, nseg, out, stream)
    torch.cuda.synchronize(dev)
    assert np.isnan(out.cpu().numpy()).all()
    t["D"][12345] = float(D[12345])
    t["E"][2 * 777] = float("inf")
    _call(P, t, ytx, nseg, out, stream)
    torch.cuda.synchronize(dev)
    assert np.isnan(out.cpu().numpy()).all()
    # no segments: g = Y'X_j, h = 0
    _call(P, t, 7.0, 0, out, stream)
    torch.cuda.synchronize(dev)
    g, h = out.cpu().numpy()
    assert g == 7.0 and h == 0.0
