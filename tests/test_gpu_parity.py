"""Parity of the CUDA path with the FP64 oracle, through the C ABI (GPU).

Per-path: final states of every pair against the oracle run with the same
Philox counters and the same uniform map (tolerances in tests/parity.py).
Reductions: the level sums against the float64 sums of the kernel's own
per-path outputs (counts bit-exact), and against the oracle's sums.
Batched launch: equal to the single-level launches.  Edge cases: empty,
single and ragged path counts, step counts that are not multiples of 4,
unstable symplectic Euler, bad arguments.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1612_07717_gb300 import workloads as W

import paper_1612_07717_gb300 as G

from parity import compare_paths, gpu_params, oracle_params, sums_from_states

pytestmark = pytest.mark.gpu

INTEGS = [G.SE, G.GL, G.BAOAB]


def _scn(integ, name):
    if name == "bl600":
        return W.bl600(integ)
    if name == "paper":
        return dict(W.PAPER, M0=40 if integ != G.SE else 40)
    if name == "wellmixed":
        d = W.well_mixed()
        if integ == G.SE:
            d["level_min"] = W.SE_LEVEL_MIN_BL600
        return d
    if name == "naive":
        d = W.bl600(integ, coupling=1)
        return d
    raise KeyError(name)


@pytest.mark.parametrize("precision", [G.FP32, G.FP64])
@pytest.mark.parametrize("name", ["bl600", "paper", "wellmixed", "naive"])
@pytest.mark.parametrize("integ", INTEGS)
def test_per_path_parity_coupled_level(integ, name, precision):
    d = _scn(integ, name)
    level = d["level_min"] + 2
    N = 4099 if precision == G.FP32 else 1031       # several blocks and a ragged tail
    dz, n_ex, gs, gf, os_ = compare_paths(d, integ, level, N, offset=17, seed=11,
                                          precision=precision)
    H = oracle_params(d).H
    assert dz <= (1e-4 if precision == G.FP32 else 1e-9) * H


@pytest.mark.parametrize("precision", [G.FP32, G.FP64])
@pytest.mark.parametrize("integ", INTEGS)
def test_per_path_parity_base_level(integ, precision):
    d = _scn(integ, "bl600")
    compare_paths(d, integ, d["level_min"], 2053, offset=0, seed=5, precision=precision)


@pytest.mark.parametrize("M0", [5, 6, 7])
@pytest.mark.parametrize("integ", [G.GL, G.BAOAB])
def test_step_counts_not_multiple_of_four(integ, M0):
    # M0 = 5 on level 1 gives 10 fine steps (a half Philox block at the end
    # of the coupled loop); M0 = 6, 7 on the base level give tails of 2, 3.
    d = dict(W.PAPER, M0=M0)
    compare_paths(d, integ, 0, 300, seed=3)
    compare_paths(d, integ, 1, 300, seed=3)


def test_large_path_indices_use_high_counter_word():
    d = W.bl600(G.BAOAB)
    compare_paths(d, G.BAOAB, 3, 300, offset=(1 << 33) + 12345, seed=9)
    compare_paths(d, G.BAOAB, 3, 300, offset=999_999_000, seed=9)


def test_trace_matches_oracle_step_by_step():
    d = W.bl600(G.GL, z0=3.0)
    pg, po = gpu_params(d, G.FP64), oracle_params(d, G.FP64)
    tf, tc = G.path_trace(3, 16, G.GL, pg, 7, path_offset=100)
    tf, tc = tf.cpu().numpy(), tc.cpu().numpy()
    for j in range(16):
        r = O.path(po, G.GL, 3, 100 + j, 7, trace=True)
        assert np.allclose(tf[j], r["trace_f"], rtol=0, atol=1e-9 * po.H)
        assert np.allclose(tc[j], r["trace_c"], rtol=0, atol=1e-9 * po.H)


@pytest.mark.parametrize("precision", [G.FP32, G.FP64])
@pytest.mark.parametrize("integ", INTEGS)
def test_reduction_equals_sums_of_own_paths(integ, precision):
    d = W.bl600(integ)
    for level in (d["level_min"], d["level_min"] + 3):
        N = 70001                                   # several hundred blocks, ragged
        pg = gpu_params(d, precision)
        gs_t, gf_t = G.level_paths(level, N, integ, pg, 13, path_offset=5)
        gs, gf = gs_t.double().cpu().numpy(), gf_t.cpu().numpy()
        ref = sums_from_states(gs, gf, d["qoi_threshold"], level > d["level_min"], precision)
        s = G.level_sums(level, N, integ, pg, 13, path_offset=5)
        assert s["n"] == ref["n"] and s["n_nonfinite"] == ref["n_nonfinite"]
        M = d["M0"] << level
        assert s["path_steps"] == N * (M + M // 2 if level > d["level_min"] else M)
        got = np.array(s["sum"])
        assert np.array_equal(got[1], ref["sum"][1])            # indicator counts: exact
        assert np.allclose(got[0], ref["sum"][0], rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("integ", INTEGS)
def test_level_means_agree_with_oracle_within_3_se(integ):
    d = W.bl600(integ)
    pg, po = gpu_params(d), oracle_params(d)
    for level in (d["level_min"], d["level_min"] + 1, d["level_min"] + 3):
        N = 20000
        g = G.level_sums(level, N, integ, pg, 21)
        o = O.level_sums(po, integ, level, N, 0, 21)
        for q in range(2):
            n = o["n"]
            mo, vo = o["sum"][q][0] / n, o["sum"][q][1] / n - (o["sum"][q][0] / n) ** 2
            mg = g["sum"][q][0] / g["n"]
            se = math.sqrt(max(vo, 1e-30) / n)
            assert abs(mg - mo) <= 3 * se + 1e-12, (level, q, mg, mo, se)
            if q == 0:
                # same random numbers: far tighter than 3 SE
                assert abs(mg - mo) <= 1e-4 * po.H


def test_offset_split_composes():
    d = W.bl600(G.GL)
    pg = gpu_params(d)
    a = G.level_sums(4, 30000, G.GL, pg, 4, path_offset=0)
    b1 = G.level_sums(4, 12345, G.GL, pg, 4, path_offset=0)
    b2 = G.level_sums(4, 30000 - 12345, G.GL, pg, 4, path_offset=12345)
    assert a["n"] == b1["n"] + b2["n"]
    assert np.array_equal(np.array(a["sum"][1]), np.array(b1["sum"][1]) + np.array(b2["sum"][1]))
    assert np.allclose(a["sum"][0], np.array(b1["sum"][0]) + np.array(b2["sum"][0]), rtol=1e-12)


@pytest.mark.parametrize("precision", [G.FP32, G.FP64])
@pytest.mark.parametrize("integ", INTEGS)
def test_multilevel_launch_equals_single_levels(integ, precision):
    d = W.bl600(integ, L_max=12)
    pg = gpu_params(d, precision)
    lm = d["level_min"]
    reqs = [(lm, 0, 200000), (lm + 1, 0, 50000), (lm + 2, 1000, 20001), (lm + 4, 7, 3001)]
    got = G.multilevel_sums(reqs, integ, pg, 31)
    for (level, first, count), g in zip(reqs, got):
        s = G.level_sums(level, count, integ, pg, 31, path_offset=first)
        assert g["n"] == s["n"] and g["path_steps"] == s["path_steps"]
        assert np.array_equal(np.array(g["sum"][1]), np.array(s["sum"][1]))
        assert np.allclose(g["sum"][0], s["sum"][0], rtol=1e-11)


def test_multilevel_is_deterministic_across_runs():
    d = W.bl600(G.BAOAB)
    pg = gpu_params(d)
    reqs = [(l, 0, n) for l, n in W.schedule_c4(levels=9, n0=2e6)]
    a = G.multilevel_sums(reqs, G.BAOAB, pg, 1)
    b = G.multilevel_sums(reqs, G.BAOAB, pg, 1)
    for x, y in zip(a, b):
        assert x == y                                # bitwise: fixed-order item reduction


def test_empty_and_single_path():
    d = W.bl600(G.GL)
    pg = gpu_params(d)
    s = G.level_sums(3, 0, G.GL, pg, 1)
    assert s["n"] == 0 and np.all(np.array(s["sum"]) == 0)
    s1 = G.level_sums(3, 1, G.GL, pg, 1, path_offset=77)
    gs, gf = G.level_paths(3, 1, G.GL, pg, 1, path_offset=77)
    zf, zc = float(gs[0, 0]), float(gs[0, 2])
    assert s1["n"] == 1 and s1["sum"][0][0] == pytest.approx(zf - zc, abs=1e-6)


def test_unstable_se_is_refused_then_flagged():
    d = W.bl600(G.SE, level_min=0)
    pg = gpu_params(d)
    with pytest.raises(G.MLMCError) as e:
        G.level_sums(2, 1000, G.SE, pg, 1)
    assert e.value.code == G.EUNSTABLE
    pu = gpu_params(d, allow_unstable=1)
    s = G.level_sums(2, 2000, G.SE, pu, 1)
    o = O.level_sums(oracle_params(d), O.SE, 2, 2000, 0, 1)
    assert s["n_nonfinite"] > 0 and o["n_nonfinite"] > 0
    assert s["n"] + s["n_nonfinite"] == 2000


def test_invalid_arguments_are_rejected():
    d = W.bl600(G.GL)
    for bad in (dict(u_star=-1.0), dict(eps_reg_frac=0.0), dict(T=0.0), dict(M0=0),
                dict(eps_reg_frac=0.7), dict(w0_mode=3), dict(z0=-1.0)):
        with pytest.raises(G.MLMCError) as e:
            G.level_sums(2, 10, G.GL, gpu_params(d, **bad), 1)
        assert e.value.code == G.EINVAL
    with pytest.raises(G.MLMCError):
        G.level_sums(2, 10, 7, gpu_params(d), 1)
    pg = gpu_params(d)
    ws = G.Workspace(pg)
    ws.nbytes = 1024
    with pytest.raises(G.MLMCError) as e:
        G.level_sums(2, 10, G.GL, pg, 1, workspace=ws)
    assert e.value.code == G.EWORKSPACE


@pytest.mark.parametrize("precision", [G.FP64, G.FP32])
def test_adaptive_estimate_matches_oracle_driver(precision):
    d = W.bl600(G.GL, L_max=8, n_init=2000)
    pg, po = gpu_params(d, precision), oracle_params(d, precision)
    eps = 600 * 2.0 ** -8
    g = G.estimate(eps, G.GL, pg, 3)
    o = O.estimate(po, O.GL, eps, seed=3)
    assert g["L"] == o["L"] and g["converged"] == o["converged"] == 1
    if precision == G.FP64:
        assert g["N"] == o["N"]
        assert g["estimate"][0] == pytest.approx(o["estimate"][0], rel=1e-10)
    else:
        for a, b in zip(g["N"], o["N"]):
            assert abs(a - b) <= max(2, 1e-3 * b)
        se = math.sqrt(o["est_variance"][0])
        assert abs(g["estimate"][0] - o["estimate"][0]) < 1e-4 * 600 + 0.1 * se


def test_stmc_estimate_reaches_its_sample_size():
    d = W.bl600(G.SE, precision=G.FP64)
    pg = gpu_params(d, G.FP64)
    eps = 600 * 2.0 ** -6
    r = G.stmc_estimate(eps, 6, G.SE, pg, 1, n_pilot=4000)
    assert r["est_variance"][0] <= 0.5 * eps ** 2 * 1.02
    assert r["N"][0] >= 4000
