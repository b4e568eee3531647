"""Host logic of the team-size autotuner: the queue simulation and the greedy assignment."""
import pytest

import __graft_entry__

__graft_entry__._build_module().build()
from paper_1208_0945_gb300.autotune import CostModel, assign, library_order, makespan


@pytest.fixture
def model():
    return CostModel(lat_us={1: 2.0, 2: 2.5, 4: 3.0, 8: 3.5, 16: 4.0, 32: 4.5, 64: 5.0, 128: 5.5},
                     c_us_per_nnz=0.002, capacity=152)


def test_makespan_of_independent_single_cta_fits(model):
    fits = [(100, 10_000, 1_000)] * 10
    t = model.cycle_us(100, 10_000, 1)
    assert makespan(fits, [1] * 10, model) == pytest.approx(t)
    # more fits than CTAs: two rounds back to back
    assert makespan(fits, [1] * 10, model, capacity=5) == pytest.approx(2 * t)


def test_team_waits_for_its_ctas_to_free_up(model):
    fits = [(10, 1_000_000, 0), (10, 1_000, 0)]
    S = [3, 3]
    t0 = model.cycle_us(10, 1_000_000, 3)
    t1 = model.cycle_us(10, 1_000, 3)
    # capacity 4: the second team needs three CTAs, only one is free until the first ends
    assert makespan(fits, S, model, capacity=4) == pytest.approx(t0 + t1)


def test_library_order_is_longest_first():
    fits = [(10, 100, 10), (500, 10_000_000, 100_000), (50, 1000, 100)]
    assert library_order(fits, [1, 1, 1]) == [1, 2, 0]


def test_assign_grows_the_big_fit_and_never_overshoots(model):
    fits = [(500, 50_000_000, 1_000_000)] + [(500, 20_000, 2_000)] * 40
    S = assign(fits, model)
    assert S[0] > 8 and all(s >= 1 for s in S)
    assert makespan(fits, S, model) < makespan(fits, [1] * len(fits), model)
    assert max(S) <= model.capacity


def test_assign_is_monotone_in_load(model):
    small = assign([(200, 100_000, 10_000)] * 4, model)
    big = assign([(200, 100_000, 10_000)] * 400, model)
    assert sum(small) / 4 >= sum(big) / 400


def test_tune_launch_takes_the_fastest_setting_of_each_knob():
    """The coordinate search over the launch knobs with a made-up cost: every knob is set to its
    fastest value given the earlier ones, each setting is probed once, and the result is the
    fastest probe."""
    from paper_1208_0945_gb300.autotune import tune_launch

    def cost(opts):
        t = 10.0
        t += {16: 0.0, 8: 1.0, -1: 3.0}[opts.get("cluster_ctas", 16)]
        t += {8192: 0.5, 16384: 0.0, 65536: 2.0}.get(opts.get("cluster_max_nnz", 16384), 0.0)
        t += {512: 0.0, 384: 0.7, 256: 1.5}[opts.get("threads_per_block", 512)]
        return t

    calls = []
    ch = tune_launch(None, timer=lambda d, o: calls.append(dict(o)) or cost(o))
    assert ch.options == {"cluster_ctas": 16, "cluster_max_nnz": 16384, "threads_per_block": 512}
    assert ch.kernel_ms == min(t for _, t in ch.trials) == cost(ch.options)
    keys = [tuple(sorted(o.items())) for o in calls]
    assert len(keys) == len(set(keys))                      # no setting probed twice
    assert len(calls) == 3 + 3 + 3                           # one probe per setting of each knob


def test_tune_launch_without_clusters_tunes_the_narrow_knobs():
    from paper_1208_0945_gb300.autotune import tune_launch

    def cost(opts):
        t = {16: 5.0, 8: 6.0, -1: 1.0}[opts["cluster_ctas"]]
        t += {512: 0.2, 1024: 0.0, 2048: 0.3}.get(opts.get("narrow_max_nnz", 1024), 0.0)
        t += {1: 0.4, 4: 0.1, 8: 0.0}.get(opts.get("narrow_group_max", 8), 0.0)
        t += {512: 0.0, 384: 0.1, 256: 0.2}[opts.get("threads_per_block", 512)]
        return t

    ch = tune_launch(None, timer=lambda d, o: cost(o))
    assert ch.options == {"cluster_ctas": -1, "narrow_max_nnz": 1024, "narrow_group_max": 8, "threads_per_block": 512}
    assert not any("cluster_max_nnz" in o for o, _ in ch.trials)
