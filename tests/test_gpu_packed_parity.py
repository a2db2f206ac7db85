"""Pair-by-pair parity of the kernels the batched launches reduce (GPU).

The benchmark's launch runs the packed kernel (two path pairs per thread on
FFMA2 / FMUL2 / FADD2, tuning variants 12 and 13).  Its path code is run here
through ``mlmc_level_paths_variant_async``, which writes each pair's final
state from that variant's own translation unit and lane code (thread g takes
pairs 2g and 2g + 1; the last lane of an odd count is computed and
discarded), and compared with the FP64 oracle on the same Philox counters
(Section 3.3: Eqs. MethodSymplecticEuler, MethodSymplecticEulerOU and
MethodBAOAB; the coupled increments of Eqs. euler_coupled_treatment and
splitting_coupled_treatment), with the tolerances and the near-tie rule of
tests/parity.py: |dz| <= 1e-4 H per pair.

Every variant must also give the same pairs bit for bit (the packed lanes
repeat the scalar operations in the same order), and the batched launch's
sums must be the FP64 sums of those pairs.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1612_07717_gb300 import autotune
from paper_1612_07717_gb300 import workloads as W

import paper_1612_07717_gb300 as G

from parity import compare_paths, gpu_params, oracle_params, sums_from_states

pytestmark = pytest.mark.gpu

INTEGS = [G.SE, G.GL, G.BAOAB]
PACKED = [12, 13]


def _scn(integ, name):
    if name == "bl600":
        return W.bl600(integ)
    if name == "paper":
        return dict(W.PAPER)
    if name == "wellmixed":
        d = W.well_mixed()
        if integ == G.SE:
            d["level_min"] = W.SE_LEVEL_MIN_BL600
        return d
    if name == "naive":
        return W.bl600(integ, coupling=1)
    raise KeyError(name)


@pytest.mark.parametrize("variant", PACKED)
@pytest.mark.parametrize("name", ["bl600", "paper", "wellmixed", "naive"])
@pytest.mark.parametrize("integ", INTEGS)
def test_packed_pairs_match_oracle(integ, name, variant):
    d = _scn(integ, name)
    level = d["level_min"] + 2
    # an odd count spanning several blocks: the last thread's second lane is discarded
    dz, n_ex, gs, gf, os_ = compare_paths(d, integ, level, 4099, offset=17, seed=11,
                                          variant=variant)
    assert dz <= 1e-4 * oracle_params(d).H


@pytest.mark.parametrize("variant", PACKED)
@pytest.mark.parametrize("integ", INTEGS)
def test_packed_base_level_and_odd_counts(integ, variant):
    d = W.bl600(integ)
    for N in (1, 2, 3, 513, 2053):
        compare_paths(d, integ, d["level_min"], N, offset=N, seed=5, variant=variant)


@pytest.mark.parametrize("variant", PACKED)
def test_packed_large_path_indices(variant):
    d = W.bl600(G.BAOAB)
    compare_paths(d, G.BAOAB, 3, 301, offset=(1 << 33) + 12345, seed=9, variant=variant)
    # a pair straddling 2^32: its two lanes differ in the counter's high word
    compare_paths(d, G.BAOAB, 3, 64, offset=(1 << 32) - 31, seed=9, variant=variant)


@pytest.mark.parametrize("M0", [5, 6, 7])
@pytest.mark.parametrize("integ", [G.GL, G.BAOAB])
def test_packed_step_counts_not_multiple_of_four(integ, M0):
    d = dict(W.PAPER, M0=M0)
    compare_paths(d, integ, 0, 301, seed=3, variant=13)
    compare_paths(d, integ, 1, 301, seed=3, variant=13)


def test_every_level_of_the_benchmark_launch_matches_oracle():
    # the benchmark's kernel (the autotuner's variant for BAOAB) on every level
    # 0..12 of its schedule: the first pairs and the last pairs of each level
    autotune.apply()
    d = W.bl600(G.BAOAB)
    for level, n_l in W.schedule_c4(levels=13, n0=1e9):
        N = 1027 if level <= 8 else 257
        compare_paths(d, G.BAOAB, level, N, offset=0, seed=1, variant=0)
        compare_paths(d, G.BAOAB, level, N, offset=n_l - N, seed=1, variant=0)


def _bits(states):
    a = states.cpu().numpy()
    return a.view(np.uint32 if a.dtype == np.float32 else np.uint64)


@pytest.mark.parametrize("precision", [G.FP32, G.FP64])
@pytest.mark.parametrize("integ", INTEGS)
def test_all_variants_give_the_same_pairs_bit_for_bit(integ, precision):
    d = W.well_mixed() if integ != G.SE else dict(W.well_mixed(),
                                                  level_min=W.SE_LEVEL_MIN_BL600)
    p = gpu_params(d, precision)
    variants = (1, 3, 4, 12, 13) if precision == G.FP32 else (1,)
    for level in (d["level_min"], d["level_min"] + 1, d["level_min"] + 4):
        for N, off in ((5001, 3), (1, 77)):
            ref_s, ref_f = G.level_paths(level, N, integ, p, 21, path_offset=off)
            ref_bits = _bits(ref_s)
            for v in variants + (0,):
                s, f = G.level_paths(level, N, integ, p, 21, path_offset=off, variant=v)
                assert np.array_equal(_bits(s), ref_bits), (level, v)
                assert np.array_equal(f.cpu().numpy(), ref_f.cpu().numpy()), (level, v)


@pytest.mark.parametrize("variant", PACKED)
@pytest.mark.parametrize("integ", INTEGS)
def test_packed_batched_sums_are_the_sums_of_its_pairs(integ, variant):
    # a few long pairs beside many short ones: the plan runs the finest
    # request one pair per thread (its pairs are long against a thread's
    # share of the launch) and the coarsest two per thread; either way the
    # sums are the FP64 sums of the pairs the variant's own lanes compute
    d = W.bl600(integ)
    lm = d["level_min"]
    p = gpu_params(d)
    saved = autotune.get_tuning(integ, G.FP32)
    reqs = [(lm + 6, 3, 3001), (lm + 1, 0, 200001), (lm, 7, 1000003)]
    try:
        autotune.set_tuning(integ, G.FP32, variant, 32, 0)
        grid = G.device_info()["sms"] * {12: 2, 13: 3}[variant]
        plan = G.multilevel_plan(reqs, integ, p, grid)
        assert [e["single"] for e in plan] == [1, 0, 0]
        got = G.multilevel_sums(reqs, integ, p, 13)
        for (level, first, count), g in zip(reqs, got):
            s, f = G.level_paths(level, count, integ, p, 13, path_offset=first,
                                 variant=variant)
            ref = sums_from_states(s.double().cpu().numpy(), f.cpu().numpy(),
                                   d["qoi_threshold"], level > lm, G.FP32)
            assert g["n"] == ref["n"] and g["n_nonfinite"] == ref["n_nonfinite"]
            assert np.array_equal(np.array(g["sum"][1]), ref["sum"][1])
            assert np.allclose(g["sum"][0], ref["sum"][0], rtol=1e-11, atol=1e-9)
    finally:
        autotune.set_tuning(integ, G.FP32, saved["variant"], saved["items_per_block"],
                            saved["blocks_per_sm"])


def test_variant_argument_is_checked():
    d = W.bl600(G.GL)
    with pytest.raises(G.MLMCError) as e:
        G.level_paths(2, 10, G.GL, gpu_params(d), 1, variant=2)
    assert e.value.code == G.EINVAL
    with pytest.raises(G.MLMCError) as e:
        G.level_paths(2, 10, G.GL, gpu_params(d, G.FP64), 1, variant=13)
    assert e.value.code == G.EINVAL
