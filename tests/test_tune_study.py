"""The autotuner's cost-model study runs on the committed GB300 cache without a GPU.

The cost model (tune.model_flags) picks the tensor-core kernel's knobs from the element
matrix's size alone; the study compares its choice, and the library's built-in default, with
the fastest candidate the tuner timed for every (form, degree, cell, precision).
"""

import pytest

from paper_1407_0904_gb300 import tune
import paper_1407_0904_gb300 as coffee


def test_study_covers_every_tuned_entry_and_the_model_is_close():
    entries = tune.load_cache(gpu="")
    if not entries:
        pytest.skip("no tuned cache committed")
    rows = tune.study(entries, log=lambda *a: None)
    assert len(rows) == len(entries)
    assert all(r["model_regret"] is not None for r in rows)  # the model's choice was a timed candidate
    mean = lambda xs: sum(xs) / len(xs)
    assert mean([r["model_regret"] for r in rows]) <= mean([r["default_regret"] for r in rows])


@pytest.mark.parametrize("n,flags", [(9, coffee.FLAG_CELL_LANES), (64, coffee.FLAG_CELL_LANES),
                                     (100, 0), (225, coffee.FLAG_SUBTILE_64), (256, coffee.FLAG_SUBTILE_64),
                                     (400, 0), (1225, 0)])
def test_model_rules(n, flags):
    assert tune.model_flags(n) == flags


@pytest.mark.parametrize("n,flags", [(9, coffee.FLAG_CUDA_CORES), (36, coffee.FLAG_CUDA_CORES),
                                     (100, coffee.FLAG_TENSOR_CORES)])
def test_model_rules_with_the_cuda_core_kernel(n, flags):
    assert tune.model_flags(n, cuda_cores=True) == flags


def test_batch_costs_prefer_in_batch_tile_times(monkeypatch):
    """BatchPlan's measured costs: the batch kernel's own per-tile time for every group when the
    cache has them, else the single-group kernel's time per 128-cell tile, else None (the plan
    then falls back to the byte model)."""
    entries = {"1/2/1/2": {"ms": 0.05, "ncells": 2 ** 19, "flags": 0},
               "0/1/0/2": {"ms": 0.03, "ncells": 2 ** 19, "flags": 0}}
    tiles = {"1/2/1/2": 0.0025, "0/1/0/2": 0.0022}
    monkeypatch.setattr(tune, "load_cache", lambda *a, **k: entries)
    monkeypatch.setattr(tune, "load_batch", lambda *a, **k: {"tile_ms": dict(tiles)})
    groups = [dict(form=1, degree=2, cell=1), dict(form=0, degree=1, cell=0)]
    assert coffee.BatchPlan.measured_costs(groups, coffee.TF32X3) == [0.0025, 0.0022]
    # a group without an in-batch time: every group takes its single-group kernel time instead
    del tiles["0/1/0/2"]
    monkeypatch.setattr(tune, "load_batch", lambda *a, **k: {"tile_ms": dict(tiles)})
    got = coffee.BatchPlan.measured_costs(groups, coffee.TF32X3)
    assert got == pytest.approx([0.05 * 128 / 2 ** 19, 0.03 * 128 / 2 ** 19])
    # a group in neither: no measured costs
    groups.append(dict(form=2, degree=4, cell=0))
    assert coffee.BatchPlan.measured_costs(groups, coffee.TF32X3) is None
    # another precision has no entries at all
    assert coffee.BatchPlan.measured_costs(groups[:1], coffee.BF16X3) is None
