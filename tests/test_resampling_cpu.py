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
