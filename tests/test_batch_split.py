"""The CTA split of the mixed batch (coffee_batch_split), host logic shared by both batch
planners: contiguous, complete, balanced to within one item's cost. No GPU needed."""
import numpy as np
import pytest

import paper_1407_0904_gb300 as coffee


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cost_split_is_contiguous_complete_and_balanced_host(seed):
    """coffee_batch_split, the rule both batch planners use: contiguous ranges covering every item
    once, and no CTA more than one item's cost above an equal share."""
    rng = np.random.default_rng(seed)
    for items, grid in ((1000, 152), (152, 152), (37, 152), (5000, 7), (1, 3)):
        cost = rng.gamma(0.5, 2.0, size=items) + (rng.random(items) < 0.02) * 50.0
        r = coffee.batch_split(cost, grid)
        assert r[0] == 0 and r[-1] == items and np.all(np.diff(r) >= 0)
        per = np.add.reduceat(np.append(cost, 0.0), r[:-1])[:grid]
        per[np.diff(r) == 0] = 0.0
        assert per.max() <= cost.sum() / grid + cost.max() + 1e-9
        assert abs(per.sum() - cost.sum()) < 1e-9 * cost.sum()


def test_cost_split_edge_cases_host():
    r = coffee.batch_split(np.ones(1000), 100)
    assert np.array_equal(r, np.arange(0, 1001, 10))  # equal costs, equal ranges
    r = coffee.batch_split(np.r_[np.ones(10), 1e6, np.ones(10)], 4)
    assert r[0] == 0 and r[-1] == 21 and np.all(np.diff(r) >= 0)
    r = coffee.batch_split(np.zeros(5), 3)  # no cost: still every item exactly once
    assert r[0] == 0 and r[-1] == 5 and np.all(np.diff(r) >= 0)
    assert np.array_equal(coffee.batch_split(np.zeros(0), 4), np.zeros(5, dtype=np.int64))
    for bad_cost, grid in ((np.array([1.0, -1.0]), 2), (np.array([np.nan]), 2), (np.ones(3), 0)):
        with pytest.raises(coffee.CoffeeError):
            coffee.batch_split(bad_cost, grid)
