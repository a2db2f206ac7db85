"""The batched launch's work-item planner (CPU: ``mlmc_multilevel_plan`` makes
no device call).

The plan must cover every requested pair exactly once, in whole passes of a
256-thread block over its pairs, with the finest level first (largest cost
per pair first, so the longest pairs start at once).  On a packed kernel (two
pairs per thread) a request runs one pair per thread when one of its pairs
alone is at least a quarter of a thread's average work: the rule is restated
here from level sizes (M0 2^l steps; a coupled pair also takes the coarse
path's half as many) and checked against the library's decisions.
"""
import pytest

import paper_1612_07717_gb300 as G
from paper_1612_07717_gb300 import autotune as A
from paper_1612_07717_gb300 import workloads as W

BLOCK = 256


def _steps_per_pair(d, level):
    M = d["M0"] << level
    return M + M // 2 if level > d["level_min"] else M


@pytest.fixture
def tuning():
    saved = {(i, p): A.get_tuning(i, p) for i in (G.SE, G.GL, G.BAOAB) for p in (G.FP32, G.FP64)}
    yield A.set_tuning
    for (i, p), t in saved.items():
        A.set_tuning(i, p, t["variant"], t["items_per_block"], t["blocks_per_sm"])


def _check_cover(reqs, plan, d, packed):
    assert sorted(e["request"] for e in plan) == list(range(len(reqs)))
    levels = [reqs[e["request"]][0] for e in plan]
    assert levels == sorted(levels, reverse=True)            # finest first
    # stable among equal levels
    for a, b in zip(plan, plan[1:]):
        if reqs[a["request"]][0] == reqs[b["request"]][0]:
            assert a["request"] < b["request"]
    base = 0
    for e in plan:
        count = reqs[e["request"]][2]
        assert e["item_base"] == base
        assert e["item_paths"] % BLOCK == 0
        if packed and not e["single"]:
            assert e["item_paths"] % (2 * BLOCK) == 0
        assert (e["n_items"] - 1) * e["item_paths"] < count <= e["n_items"] * e["item_paths"]
        base += e["n_items"]
    return base


def _expected_single(reqs, d, grid):
    total = sum(n * _steps_per_pair(d, l) for l, _, n in reqs)
    share = 0.25 * total / (grid * BLOCK)
    return {k: _steps_per_pair(d, l) >= share for k, (l, _, n) in enumerate(reqs)}


@pytest.mark.parametrize("variant,grid", [(12, 304), (13, 456), (12, 152), (13, 1000)])
@pytest.mark.parametrize("integ", [G.SE, G.GL, G.BAOAB])
def test_packed_plan_covers_every_pair_and_follows_the_single_rule(tuning, integ, variant, grid):
    tuning(integ, G.FP32, variant, 32, 0)
    d = W.bl600(integ)
    p = G.make_params(d)
    lm = d["level_min"]
    for reqs in ([(l, 0, n) for l, n in W.schedule_c4(13, 1e9) if l >= lm],
                 [(lm + 6, 5, 3001), (lm + 1, 0, 200001), (lm, 17, 1000003)],
                 [(lm + 2, 0, 1), (lm, 0, 1)],
                 [(lm, 0, 4096), (lm + 3, 11, 999), (lm + 3, 0, 7)]):
        plan = G.multilevel_plan(reqs, integ, p, grid)
        _check_cover(reqs, plan, d, packed=True)
        want = _expected_single(reqs, d, grid)
        assert {e["request"]: bool(e["single"]) for e in plan} == want, reqs


def test_single_on_tail_bound_batches_only(tuning):
    # the benchmark's 13-level BAOAB batch on 152 SMs x 3 blocks: no level's
    # pair reaches a quarter of a thread's share (level 12: 49152 steps of
    # about 2.4e5 per thread) -- the whole launch stays packed
    tuning(G.BAOAB, G.FP32, 13, 32, 0)
    d = W.bl600(G.BAOAB)
    reqs = [(l, 0, n) for l, n in W.schedule_c4(13, 1e9)]
    plan = G.multilevel_plan(reqs, G.BAOAB, G.make_params(d), 456)
    assert not any(e["single"] for e in plan)
    # SE's levels 6..12 of the same schedule: 1.75e9 path-steps, about 2.2e4
    # per thread on 152 x 2 blocks, so levels 9 (6144 steps) to 12 go single
    tuning(G.SE, G.FP32, 12, 32, 0)
    d = W.bl600(G.SE)
    reqs = [(l, 0, n) for l, n in W.schedule_c4(13, 1e9) if l >= 6]
    plan = G.multilevel_plan(reqs, G.SE, G.make_params(d), 304)
    assert {reqs[e["request"]][0] for e in plan if e["single"]} == {9, 10, 11, 12}


@pytest.mark.parametrize("variant", [1, 3, 4])
def test_one_pair_kernels_never_go_single(tuning, variant):
    tuning(G.SE, G.FP32, variant, 8, 0)
    d = W.bl600(G.SE)
    reqs = [(12, 0, 1000), (6, 0, 1000000)]
    plan = G.multilevel_plan(reqs, G.SE, G.make_params(d), 608)
    _check_cover(reqs, plan, d, packed=False)
    assert not any(e["single"] for e in plan)


def test_fp64_and_adaptive_batches_never_go_single(tuning):
    d = W.bl600(G.GL)
    reqs = [(9, 0, 100), (0, 0, 100000)]
    plan = G.multilevel_plan(reqs, G.GL, G.make_params(d, precision=G.FP64), 152)
    assert not any(e["single"] for e in plan)
    tuning(G.SE, G.FP32, 12, 32, 0)
    pa = G.make_params(dict(W.PAPER, z_adapt=0.05))
    plan = G.multilevel_plan([(5, 0, 100), (0, 0, 100000)], G.SE, pa, 152)
    assert not any(e["single"] for e in plan)
    assert all(e["item_paths"] % BLOCK == 0 for e in plan)


def test_plan_rejects_bad_arguments():
    d = W.bl600(G.GL)
    p = G.make_params(d)
    with pytest.raises(G.MLMCError) as e:
        G.multilevel_plan([(1, 0, 10)], G.GL, p, 0)
    assert e.value.code == G.EINVAL
    with pytest.raises(G.MLMCError) as e:
        G.multilevel_plan([(0, 0, 10)] * 33, G.GL, p, 152)
    assert e.value.code == G.EINVAL
    with pytest.raises(G.MLMCError) as e:
        G.multilevel_plan([(0, 0, 10)], 7, p, 152)
    assert e.value.code == G.EINVAL


@pytest.mark.parametrize("integ", [G.SE, G.GL])
def test_adaptive_plan_does_not_follow_the_uniform_kernels_tuning(tuning, integ):
    # adaptive batches run their own kernel: the uniform kernel's variant and
    # item size must not change their split
    pa = G.make_params(dict(W.PAPER, z_adapt=0.05))
    reqs = [(6, 0, 20001), (3, 0, 100000), (0, 0, 400000)]
    plans = []
    for variant, ipb in ((1, 4), (12, 64), (13, 8)):
        tuning(integ, G.FP32, variant, ipb, 0)
        plans.append(G.multilevel_plan(reqs, integ, pa, 304))
    assert plans[0] == plans[1] == plans[2]
    _check_cover(reqs, plans[0], dict(W.PAPER), packed=False)


def test_huge_batches_cap_items_below_2_31_pairs_in_whole_passes(tuning):
    # 2^45 pairs need items larger than 2^31 - 1 pairs: they are capped at the
    # largest whole number of block passes below that and still cover the batch;
    # at 2^46 pairs even capped items exceed the 32768 items of one launch
    tuning(G.GL, G.FP32, 13, 32, 0)
    d = W.bl600(G.GL)
    p = G.make_params(d)
    reqs = [(0, 0, 2 ** 45)]
    plan = G.multilevel_plan(reqs, G.GL, p, 456)
    assert plan[0]["item_paths"] <= 2 ** 31 - 1
    assert plan[0]["item_paths"] >= 2 ** 31 - 2 * BLOCK
    _check_cover(reqs, plan, d, packed=True)
    with pytest.raises(G.MLMCError) as e:
        G.multilevel_plan([(0, 0, 2 ** 46)], G.GL, p, 456)
    assert e.value.code == G.EINVAL
