"""The autotuner's choice among measured configurations (host logic; the measurements themselves
are GPU work, covered in tests/test_gpu_multi.py)."""
import pytest

from paper_2506_02219_gb300 import autotune

ROWS = [
    {"leaf_size": 1, "S": 1, "schedule": 0, "ms": 10.0, "median_rel_err": 0.04},  # 10 * 0.0016 = 0.016
    {"leaf_size": 1, "S": 2, "schedule": 0, "ms": 18.0, "median_rel_err": 0.028},  # 0.0141
    {"leaf_size": 4, "S": 4, "schedule": 0, "ms": 40.0, "median_rel_err": 0.02},  # 0.016
    {"leaf_size": 4, "S": 1, "schedule": 1, "ms": 25.0, "median_rel_err": 0.05},  # 0.0625
]


def test_without_a_target_the_least_time_times_error_squared():
    assert autotune.select(ROWS) is ROWS[1]


def test_with_a_target_the_fastest_row_that_meets_it():
    assert autotune.select(ROWS, 0.03) is ROWS[1]
    assert autotune.select(ROWS, 0.045) is ROWS[0]
    assert autotune.select(ROWS, 0.02) is ROWS[2]  # met exactly


def test_an_unreachable_target_takes_the_most_accurate_row():
    assert autotune.select(ROWS, 0.001) is ROWS[2]


def test_ties_keep_table_order_and_empty_tables_are_rejected():
    rows = [dict(ROWS[0]), dict(ROWS[0])]
    assert autotune.select(rows) is rows[0]
    with pytest.raises(ValueError):
        autotune.select([])
