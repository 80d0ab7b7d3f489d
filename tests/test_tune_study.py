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
