"""The autotuner's choice rule (CPU): the first combination in sweep order
within 1 % of the fastest."""
from paper_1612_07717_gb300 import autotune as A


def test_first_within_tolerance_in_sweep_order():
    rows = [(2.70, 1, 4), (2.718, 1, 8), (2.74, 3, 16), (2.741, 3, 64), (2.5, 13, 32)]
    assert A.select(rows) == (2.718, 1, 8)          # 0.84 % below the best
    assert A.select(rows, tolerance=0.0) == (2.741, 3, 64)
    assert A.select([(1.0, 13, 32)]) == (1.0, 13, 32)
