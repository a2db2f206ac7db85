"""The autotuner's host logic (CPU): the choice rule (the first combination in
sweep order within 1 % of the fastest) and the tuned launch's schedule."""
import paper_1612_07717_gb300 as G
from paper_1612_07717_gb300 import autotune as A
from paper_1612_07717_gb300 import workloads as W


def test_first_within_tolerance_in_sweep_order():
    rows = [(2.70, 1, 4), (2.718, 1, 8), (2.74, 3, 16), (2.741, 3, 64), (2.5, 13, 32)]
    assert A.select(rows) == (2.718, 1, 8)          # 0.84 % below the best
    assert A.select(rows, tolerance=0.0) == (2.741, 3, 64)
    assert A.select([(1.0, 13, 32)]) == (1.0, 13, 32)


def test_tuning_schedule_is_the_benchmark_launch_for_level_min_0():
    for integ in (G.GL, G.BAOAB):
        assert A.tuning_schedule(integ, 1e9) == W.schedule_c4(levels=13, n0=1e9)


def test_se_tuning_schedule_matches_the_path_steps_of_levels_0_to_12():
    full = A._steps(W.schedule_c4(levels=13, n0=1e9), 0)
    se = A.tuning_schedule(G.SE, 1e9)
    assert [l for l, _ in se] == list(range(W.SE_LEVEL_MIN_BL600, 13))
    assert abs(A._steps(se, W.SE_LEVEL_MIN_BL600) / full - 1.0) < 1e-6
    # still the geometric N_l = c 10^(-l/2) of the hierarchy
    for (_, a), (_, b) in zip(se, se[1:]):
        assert abs(a / b - 10 ** 0.5) < 1e-3
    # hand count: level 6 pairs take 512 steps, level 7 pairs 1024 + 512
    assert A._steps([(6, 2), (7, 3)], 6) == 2 * 512 + 3 * 1536
