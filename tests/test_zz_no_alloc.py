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
