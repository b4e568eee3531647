"""Host logic of the resampling API (no GPU): the seeded draws and the summaries."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def R():
    import __graft_entry__
    __graft_entry__._build_module().build()
    from paper_1208_0945_gb300 import resampling
    return resampling


def test_folds_partition_the_subjects(R):
    f = R.draw_folds(1003, 10, seed=4)
    assert f.shape == (1003,) and set(np.unique(f)) == set(range(1, 11))
    sizes = np.bincount(f)[1:]
    assert sizes.max() - sizes.min() <= 1
    assert np.array_equal(f, R.draw_folds(1003, 10, seed=4))
    assert not np.array_equal(f, R.draw_folds(1003, 10, seed=5))
    with pytest.raises(ValueError):
        R.draw_folds(5, 6, seed=0)


def test_bootstrap_draws_resample_all_subjects(R):
    W = R.draw_bootstrap(500, 40, seed=9)
    assert W.shape == (40, 500) and W.dtype == np.int32 and (W >= 0).all()
    assert (W.sum(axis=1) == 500).all()
    # about 1 - 1/e of the subjects appear in a replicate
    assert abs(np.mean(W > 0) - (1 - np.exp(-1))) < 0.03
    assert np.array_equal(W, R.draw_bootstrap(500, 40, seed=9))


def test_interval_summary(R):
    b = np.array([[0.0, 1.0, -2.0], [0.0, 3.0, -2.0], [1.0, 2.0, 0.0], [0.0, 4.0, -1.0]])
    s = R.interval_summary(b, level=0.5)
    np.testing.assert_allclose(s["lower"], np.quantile(b, 0.25, axis=0))
    np.testing.assert_allclose(s["upper"], np.quantile(b, 0.75, axis=0))
    np.testing.assert_array_equal(s["p_nonzero"], [0.25, 1.0, 0.75])
    s95 = R.interval_summary(np.arange(201, dtype=float)[:, None])
    np.testing.assert_allclose([s95["lower"][0], s95["upper"][0]], [5.0, 195.0])   # 2.5% and 97.5%
    with pytest.raises(ValueError):
        R.interval_summary(b, level=1.0)
    with pytest.raises(ValueError):
        R.interval_summary(np.zeros(3))


class _FakeServer:
    """Records submissions; results carry the request's own index, completed in any order."""

    def __init__(self):
        self.outstanding, self.max_outstanding, self.closed = set(), 0, False
        self.next = 0

    def submit(self, model, alt=None, **kw):
        t = self.next
        self.next += 1
        self.outstanding.add(t)
        self.max_outstanding = max(self.max_outstanding, len(self.outstanding))
        self.kw = kw
        return t

    def wait(self, t):
        self.outstanding.discard(t)
        return {"status": 0, "ticket": t, "beta": np.array([float(t)]), "cycles": 1, "logpost": 0.0,
                "heldout_loglik": -float(t)}

    def close(self):
        self.closed = True


def test_submission_window_and_result_order(R):
    srv = _FakeServer()
    reqs = [dict(variance=float(i)) for i in range(10)]
    res = R._run(None, reqs, srv, None, 4, window=3)
    assert [r["ticket"] for r in res] == list(range(10))     # results in request order
    assert srv.max_outstanding <= 3 and not srv.outstanding
    assert not srv.closed                                      # a caller's server stays open


def test_failed_fits_are_reported(R):
    with pytest.raises(RuntimeError):
        R._check_done([{"status": 0}, {"status": -7}], "bootstrap")
    R._check_done([{"status": 0}, {"status": 1}], "bootstrap")   # not converged is kept
