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
