"""The fit server: requests over several resident datasets, admitted as room frees up and
run concurrently, must each give bit for bit what sccs_fit gives for the same dataset,
prior and options when run alone."""
import time

import numpy as np
import pytest

from synth import make_dataset

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1208_0945_gb300 as P
    return P


def _data(n, seed, J=40):
    return make_dataset(n_patients=n, eras=("geometric", 8), J=J, columns=("density_range", 0.005, 0.05),
                        n_true=3, beta_sd=0.4, seed=seed)


@pytest.fixture(scope="module")
def models(P):
    specs = [(3000, 500, 2), (20000, 501, 8), (80000, 502, 24), (150000, 503, 60)]
    ms = [P.SCCSModel(_data(n, seed), device=0, num_shards=s) for n, seed, s in specs]
    yield ms
    for m in ms:
        m.close()


def _alone(m, prior, var, **kw):
    m.set_prior(prior, var)
    return m.fit(**kw)


def _same(r, a):
    assert r["status"] == a["status"], (r["status"], a["status"])
    assert r["cycles"] == a["cycles"] and r["fp32_cycles"] == a["fp32_cycles"]
    assert r["logpost"] == a["logpost"]
    assert np.array_equal(r["beta"], a["beta"])


def test_mixed_requests_match_standalone_fits(P, models):
    priors = [("normal", 0.05), ("laplace", 0.1), ("normal", 1.0), ("laplace", 0.02), ("none", 1.0)]
    reqs = []
    for i, m in enumerate(models):
        for k, (prior, var) in enumerate(priors):
            reqs.append((m, prior, var, dict(tol=1e-12, max_cycles=200 if prior != "none" else 30)))
    alone = [_alone(m, prior, var, **kw) for m, prior, var, kw in reqs]
    with P.FitServer(device=0, max_inflight=16) as srv:
        tickets = [srv.submit(m, prior=prior, variance=var, **kw) for m, prior, var, kw in reqs]
        got = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["pending"] == 0 and st["running"] == 0
    for r, a in zip(got, alone):
        _same(r, a)
        assert r["latency_ms"] >= r["queue_ms"] >= 0.0


def test_arrivals_while_others_run(P, models):
    """Requests submitted in a stream (several copies of the same fit) all agree bit for bit."""
    m = models[2]
    a = _alone(m, "normal", 0.1, tol=1e-12, max_cycles=100)
    with P.FitServer(device=0, max_inflight=4) as srv:
        tickets = []
        for _ in range(12):
            tickets.append(srv.submit(m, prior="normal", variance=0.1, tol=1e-12, max_cycles=100))
            time.sleep(0.002)
        for t in tickets:
            _same(srv.wait(t), a)


def test_precisions_and_warm_start(P, models):
    m = models[1]
    rng = np.random.default_rng(7)
    b0 = rng.normal(0, 0.1, m.J)
    cases = [dict(precision="fp32_polish", tol=1e-12, max_cycles=200),
             dict(precision="fp32", tol=-1.0, max_cycles=6),
             dict(precision="fp64", tol=-1.0, max_cycles=5, beta0=b0)]
    alone = [_alone(m, "normal", 0.2, **kw) for kw in cases]
    with P.FitServer(device=0) as srv:
        tickets = [srv.submit(m, prior="normal", variance=0.2, **kw) for kw in cases]
        for t, a in zip(tickets, alone):
            _same(srv.wait(t), a)


def test_budget_too_small_fails_the_request(P, models):
    with P.FitServer(device=0, hbm_budget_bytes=1024) as srv:
        t = srv.submit(models[0], prior="normal", variance=1.0)
        r = srv.wait(t)
    assert r["status"] == P.sccs.E_NOMEM


def test_budget_admits_one_slot_at_a_time(P, models):
    """A budget for one fit slot serialises the requests; each still gives its standalone result."""
    m = models[1]
    a = _alone(m, "laplace", 0.1, tol=1e-12, max_cycles=100)
    with P.FitServer(device=0) as probe:
        probe.wait(probe.submit(m, prior="laplace", variance=0.1, tol=1e-12, max_cycles=100))
        one = probe.stats()["slot_bytes"]
    with P.FitServer(device=0, hbm_budget_bytes=one) as srv:
        tickets = [srv.submit(m, prior="laplace", variance=0.1, tol=1e-12, max_cycles=100) for _ in range(4)]
        seen_running = 0
        while srv.stats()["completed"] < 4:
            seen_running = max(seen_running, srv.stats()["running"])
            time.sleep(0.0005)
        assert seen_running <= 1 and srv.stats()["slot_bytes"] <= one
        for t in tickets:
            _same(srv.wait(t), a)


def test_queue_full_and_bad_tickets(P, models):
    m_long, m = models[3], models[0]
    with P.FitServer(device=0, max_inflight=1, queue_capacity=1) as srv:
        t0 = srv.submit(m_long, prior="normal", variance=1.0, tol=-1.0, max_cycles=400)
        t_end = time.perf_counter() + 5.0
        while srv.stats()["running"] != 1 and time.perf_counter() < t_end:
            time.sleep(0.0002)
        assert srv.stats()["running"] == 1
        t1 = srv.submit(m, prior="normal", variance=1.0)
        with pytest.raises(P.SCCSError) as ei:
            P.sccs_submit(srv.server, m.handle, prior="normal", variance=1.0)
        assert ei.value.code == P.sccs.E_BUSY
        r0, r1 = srv.wait(t0), srv.wait(t1)
        assert r0["status"] == P.sccs.NOT_CONVERGED and r0["cycles"] == 400
        assert r1["status"] == P.sccs.OK
        with pytest.raises(P.SCCSError):
            P.sccs_poll(srv.server, t1, m.J)   # already collected
        with pytest.raises(P.SCCSError):
            P.sccs_poll(srv.server, 999999, m.J)


def test_destroy_with_requests_outstanding(P, models):
    srv = P.FitServer(device=0, max_inflight=1)
    for _ in range(6):
        srv.submit(models[2], prior="normal", variance=1.0, tol=-1.0, max_cycles=20)
    srv.close()   # queued requests are cancelled, the running one finishes; nothing leaks or hangs
    m = models[0]
    m.set_prior("normal", 1.0)
    assert m.fit(tol=1e-10)["status"] == P.sccs.OK


def test_alternative_team_at_low_and_high_load(P):
    """A request naming two layouts of the same data runs on the larger team when the device is
    idle and on the smaller one in a burst; each result equals the standalone fit on the handle
    it ran on, bit for bit."""
    d = _data(40000, 510)
    small = P.SCCSModel(d, device=0, num_shards=6)
    large = P.SCCSModel(d, device=0, num_shards=48)
    try:
        kw = dict(prior="normal", variance=0.2, tol=1e-12, max_cycles=200)
        alone = {}
        for m in (small, large):
            m.set_prior("normal", 0.2)
            alone[m.info["num_shards"]] = m.fit(tol=1e-12, max_cycles=200)
        with P.FitServer(device=0, max_inflight=16) as srv:
            quiet = [srv.wait(srv.submit(small, alt=large, **kw)) for _ in range(3)]
            burst = [srv.submit(small, alt=large, **kw) for _ in range(12)]
            burst = [srv.wait(t) for t in burst]
        assert all(r["team"] == 48 for r in quiet)
        assert any(r["team"] == 6 for r in burst)
        for r in quiet + burst:
            a = alone[r["team"]]
            assert r["cycles"] == a["cycles"] and r["logpost"] == a["logpost"]
            assert np.array_equal(r["beta"], a["beta"])
        np.testing.assert_allclose(alone[6]["beta"], alone[48]["beta"], atol=1e-12, rtol=0)
    finally:
        small.close()
        large.close()
