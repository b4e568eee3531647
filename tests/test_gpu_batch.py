"""Batched fits: several independent fits in one persistent launch (one CTA team per fit).
Each fit must give bit for bit what it gives alone, however the batch is packed."""
import numpy as np
import pytest

import oracle
from synth import make_dataset

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1208_0945_gb300 as P
    return P


def _datasets(sizes, seed0=100, J=40):
    return [make_dataset(n_patients=n, eras=("geometric", 8), J=J, columns=("density_range", 0.005, 0.05),
                         n_true=3, beta_sd=0.4, seed=seed0 + i) for i, n in enumerate(sizes)]


def _models(P, ds, shards, priors):
    ms = []
    for d, s, (prior, var) in zip(ds, shards, priors):
        m = P.SCCSModel(d, device=0, num_shards=s)
        m.set_prior(prior, var)
        ms.append(m)
    return ms


def test_batch_equals_standalone_bitwise(P):
    ds = _datasets([2000, 5000, 20000, 60000, 150000])
    priors = [("normal", 0.01), ("normal", 0.1), ("laplace", 0.05), ("normal", 1.0), ("laplace", 0.2)]
    ms = _models(P, ds, [1, 3, 8, 16, 40], priors)
    try:
        batch = P.sccs_fit_batch([m.handle for m in ms], [m.J for m in ms], tol=1e-13, max_cycles=100)
        for m, b in zip(ms, batch):
            r = m.fit(tol=1e-13, max_cycles=100)
            assert b["status"] == r["status"] and b["cycles"] == r["cycles"]
            assert np.array_equal(r["beta"], b["beta"]) and r["logpost"] == b["logpost"]
    finally:
        for m in ms:
            m.close()


def test_batch_with_more_ctas_than_the_device_fp32_polish(P):
    """More shards than the device holds at once: CTAs take several fits' tickets in turn."""
    ds = _datasets([30000] * 6, seed0=200)
    ms = _models(P, ds, [40] * 6, [("normal", 0.1)] * 6)
    try:
        batch = P.sccs_fit_batch([m.handle for m in ms], [m.J for m in ms], precision="fp32_polish",
                                 tol=-1.0, max_cycles=5)
        for m, b in zip(ms, batch):
            r = m.fit(precision="fp32_polish", tol=-1.0, max_cycles=5)
            assert b["fp32_cycles"] == r["fp32_cycles"] > 0
            assert np.array_equal(r["beta"], b["beta"])
    finally:
        for m in ms:
            m.close()


def test_batch_against_oracle(P):
    ds = _datasets([3000, 12000], seed0=300)
    ms = _models(P, ds, [2, 6], [("normal", 0.1), ("normal", 0.5)])
    try:
        batch = P.sccs_fit_batch([m.handle for m in ms], [m.J for m in ms], tol=-1.0, max_cycles=3)
        for d, b, var in zip(ds, batch, (0.1, 0.5)):
            ref = oracle.Problem.from_data(d).fit(prior="normal", variance=var, fixed_cycles=3)
            np.testing.assert_allclose(b["beta"], ref["beta"], atol=1e-11, rtol=0)
            assert abs(b["logpost"] - ref["logpost"]) <= 1e-12 * abs(ref["logpost"])
    finally:
        for m in ms:
            m.close()


def test_many_small_fits_share_ctas(P):
    """300 one- to three-CTA fits: every CTA runs many fits in turn, each as it runs alone."""
    ds = _datasets([1500 + 37 * i for i in range(300)], seed0=1000, J=12)
    ms = _models(P, ds, [1 + i % 3 for i in range(300)], [("normal", (0.05, 0.5, 2.0)[i % 3]) for i in range(300)])
    try:
        batch = P.sccs_fit_batch([m.handle for m in ms], [m.J for m in ms], tol=1e-12, max_cycles=60)
        for i in (0, 1, 2, 57, 150, 298, 299):
            r = ms[i].fit(tol=1e-12, max_cycles=60)
            b = batch[i]
            assert b["status"] == r["status"] and b["cycles"] == r["cycles"]
            assert np.array_equal(r["beta"], b["beta"]) and r["logpost"] == b["logpost"]
    finally:
        for m in ms:
            m.close()


def test_repeated_batches_replay_with_new_priors(P):
    """The second call over the same handles replays the cached plan with the new priors."""
    ds = _datasets([4000, 9000, 25000], seed0=400)
    ms = _models(P, ds, [2, 4, 8], [("normal", 0.1)] * 3)
    try:
        for var in (0.1, 1.0, 0.01):
            for m in ms:
                m.set_prior("laplace" if var == 1.0 else "normal", var)
            batch = P.sccs_fit_batch([m.handle for m in ms], [m.J for m in ms], tol=1e-12, max_cycles=80)
            for m, b in zip(ms, batch):
                r = m.fit(tol=1e-12, max_cycles=80)
                assert np.array_equal(r["beta"], b["beta"]) and r["cycles"] == b["cycles"]
        # warm start from the state the last standalone fit left
        batch = P.sccs_fit_batch([m.handle for m in ms], [m.J for m in ms], warm_start=True, tol=-1.0, max_cycles=2)
        for m, b in zip(ms, batch):
            r = m.fit(warm_start=True, tol=-1.0, max_cycles=2)
            # the standalone warm fit starts where the batch left off: both are at the MAP
            assert np.allclose(r["beta"], b["beta"], atol=1e-9)
    finally:
        for m in ms:
            m.close()


def test_destroyed_handle_drops_cached_plans(P):
    ds = _datasets([3000, 6000], seed0=500)
    for rep in range(3):
        ms = _models(P, ds, [1, 2], [("normal", 0.5)] * 2)
        try:
            batch = P.sccs_fit_batch([m.handle for m in ms], [m.J for m in ms], tol=1e-12, max_cycles=50)
            r = ms[1].fit(tol=1e-12, max_cycles=50)
            assert np.array_equal(r["beta"], batch[1]["beta"])
        finally:
            for m in ms:
                m.close()


def test_batch_with_genkin_rule_equals_standalone(P):
    ds = _datasets([5000, 20000], seed0=600)
    ms = _models(P, ds, [2, 6], [("normal", 0.2), ("laplace", 0.1)])
    try:
        batch = P.sccs_fit_batch([m.handle for m in ms], [m.J for m in ms], tol_mode="genkin_xbeta", tol=1e-7,
                                 max_cycles=100)
        for m, b in zip(ms, batch):
            r = m.fit(tol_mode="genkin_xbeta", tol=1e-7, max_cycles=100)
            assert b["cycles"] == r["cycles"] and np.array_equal(r["beta"], b["beta"])
    finally:
        for m in ms:
            m.close()
