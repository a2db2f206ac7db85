"""Adaptive, non-nested timesteps on the GPU against the oracle (Section 7.2
and 7.3 of the paper).

* FP64 paths: per pair the final states equal the oracle's to 1e-9 H and the
  step counts are equal (a pair may be exempt only if the oracle met a step
  decision with a margin below 1e-12: X_n within 1e-12 H of X_adapt, or
  1024 lambda(X_adapt) / lambda(X_n) within 1e-9 of an integer).  Level sums
  agree with the oracle's sums over the same pairs.
* FP32 paths: a step decision is a threshold, so where the FP32 position
  and lambda differ from the FP64 ones by more than the decision margin the
  pair can take another merged grid.  Pairs whose oracle decisions all had a
  margin above 1e-5 follow the oracle step for step (equal step counts,
  final position within 1e-4 H up to reflection near-ties); level means and
  mean step counts agree with the oracle's within their sampling error.
* The batched launch equals the single-level launch; the host estimator
  converges with the measured cost and reaches the paper's mean position;
  adaptive SE runs on levels where uniform SE is refused as unstable.
* Section 7.3 in its scenario (X_adapt = 0.05), with 1e6 pairs per level:
  Var[Y_l] falls about 4x per level, adaptivity lowers it at a given h_l, the
  SE bias shrinks about 6x and the GL bias grows about 3x.
* Entry points without adaptive support refuse it.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1612_07717_gb300 import workloads as W

import paper_1612_07717_gb300 as G

from parity import gpu_params, oracle_params

pytestmark = pytest.mark.gpu

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
XA = GOLDEN["adaptive_bias_ratio"]["X_adapt"]

CASES = [
    (G.SE, dict(W.bl600(G.SE), z_adapt=30.0), 7),        # coupled, 1024 + 512 steps
    (G.SE, dict(W.bl600(G.SE), z_adapt=30.0), 6),        # level_min: fine path only
    (G.GL, dict(W.bl600(G.GL), z_adapt=30.0), 3),
    (G.GL, dict(W.PAPER, z_adapt=XA), 2),
    (G.SE, dict(W.PAPER, z_adapt=XA, coupling=1), 2),    # all S = 1
]


def _run_both(integ, d, level, N, offset, seed, precision):
    pg = gpu_params(d, precision)
    po = oracle_params(d, precision)
    states, flags, steps = G.level_paths(level, N, integ, pg, seed, path_offset=offset, steps=True)
    gs = states.double().cpu().numpy()
    gf = flags.cpu().numpy()
    gst = steps.cpu().numpy()
    os_, of, ost, tie = O.paths(po, integ, level, N, offset, seed, extra=True)
    return po.H, gs, gf, gst, os_, of, ost, tie


@pytest.mark.parametrize("case", range(len(CASES)))
def test_fp64_pairs_equal_the_oracle(case):
    integ, d, level = CASES[case]
    N = 2000
    H, gs, gf, gst, os_, of, ost, tie = _run_both(integ, d, level, N, 3, 17, G.FP64)
    assert gf.sum() == 0 and of.sum() == 0
    exempt = tie[:, 0] < 1e-12
    assert exempt.sum() <= max(2, N // 100)
    ok = ~exempt
    assert np.array_equal(gst[ok], ost[ok]), "step counts differ"
    dz = np.abs(gs[ok] - os_[ok])
    assert dz[:, [0, 2]].max() <= 1e-9 * H, dz.max(axis=0)
    assert dz[:, [1, 3]].max() <= 1e-9 * max(1.0, np.abs(os_[:, [1, 3]]).max())


@pytest.mark.parametrize("case", [0, 2, 3])
def test_fp64_level_sums_equal_the_oracle(case):
    integ, d, level = CASES[case]
    N = 20000
    s = G.level_sums(level, N, integ, gpu_params(d, G.FP64), 5, path_offset=100)
    o = O.level_sums(oracle_params(d, G.FP64), integ, level, N, 100, 5)
    assert s["n"] == o["n"] == N
    assert s["path_steps"] == o["path_steps"]
    for q in range(2):
        assert np.allclose(s["sum"][q], o["sum"][q], rtol=1e-9, atol=1e-9 * N), q


@pytest.mark.parametrize("case", range(len(CASES)))
def test_fp32_pairs_with_clear_step_decisions_follow_the_oracle(case):
    integ, d, level = CASES[case]
    N = 2000
    H, gs, gf, gst, os_, of, ost, tie = _run_both(integ, d, level, N, 3, 17, G.FP32)
    assert gf.sum() == 0 and of.sum() == 0
    calm = tie[:, 0] > 1e-5
    assert calm.mean() > 0.2, calm.mean()
    assert np.array_equal(gst[calm], ost[calm]), "step counts differ"
    dz = np.abs(gs[calm][:, [0, 2]] - os_[calm][:, [0, 2]]).max(axis=1)
    far = dz > 1e-4 * H
    assert far.sum() <= max(2, calm.sum() // 1000), (far.sum(), np.sort(dz)[-5:] / H)


@pytest.mark.parametrize("case", [0, 2, 3])
def test_fp32_level_statistics_match_the_oracle(case):
    integ, d, level = CASES[case]
    N = 40000
    s = G.level_sums(level, N, integ, gpu_params(d, G.FP32), 5)
    o = O.level_sums(oracle_params(d, G.FP32), integ, level, N, 0, 5)
    assert s["n"] == o["n"] == N
    for q in range(2):
        for k in (0, 2, 4):              # sums of Y, P_f, P_c
            sq = k + 1
            var = max(o["sum"][q][sq] / N - (o["sum"][q][k] / N) ** 2, 1e-30)
            se = math.sqrt(2 * var / N)
            assert abs(s["sum"][q][k] / N - o["sum"][q][k] / N) <= 4 * se + 1e-12, (q, k)
    assert abs(s["path_steps"] / o["path_steps"] - 1) < 0.01


def test_batched_launch_equals_single_level_launches():
    integ = G.GL
    d = dict(W.bl600(integ), z_adapt=30.0)
    pg = gpu_params(d)
    reqs = [(5, 0, 3001), (2, 11, 40000), (0, 0, 100000)]
    got = G.multilevel_sums(reqs, integ, pg, 7)
    for (l, f, n), g in zip(reqs, got):
        s = G.level_sums(l, n, integ, pg, 7, path_offset=f)
        assert g["n"] == s["n"] and g["path_steps"] == s["path_steps"]
        assert np.array_equal(np.array(g["sum"][1]), np.array(s["sum"][1]))
        assert np.allclose(g["sum"][0], s["sum"][0], rtol=1e-11)


def test_estimate_with_adaptive_se_reaches_the_paper_value():
    d = dict(W.PAPER, z_adapt=XA, n_init=10000, L_max=9)
    p = gpu_params(d)
    eps = 2e-4
    r = G.estimate(eps, G.SE, p, 31)
    assert r["converged"] == 1
    g = GOLDEN["mean_position"]
    rmse = math.sqrt(r["est_variance"][0]) + eps / math.sqrt(2)
    assert abs(r["estimate"][0] - g["value"]) <= 3 * rmse + g["tolerance"]
    uniform_cost = sum(n * ((40 << l) * 3 // 2 if l > 0 else 40)
                       for l, n in enumerate(r["N"]))
    assert r["total_path_steps"] > uniform_cost


def test_adaptive_se_runs_where_uniform_se_is_refused():
    d = W.bl600(G.SE, level_min=0)
    with pytest.raises(G.MLMCError) as e:
        G.level_sums(2, 1000, G.SE, gpu_params(d), 1)
    assert e.value.code == G.EUNSTABLE
    # X_adapt with 2h lambda(X_adapt) = 1 at level 2 (2h = 37.5 s)
    po = O.make_params(d)
    lo, hi = 1.0, 300.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if 37.5 * O.coefficients(po, mid)[3] > 1 else (lo, mid)
    s = G.level_sums(2, 100000, G.SE, gpu_params(dict(d, z_adapt=hi)), 1)
    assert s["n_nonfinite"] == 0 and s["n"] == 100000


def _stats(p, integ, level, N, seed):
    s = G.level_sums(level, N, integ, p, seed)
    n = s["n"]
    m = s["sum"][0][0] / n
    v = s["sum"][0][1] / n - m * m
    return m, v, math.sqrt(v / n)


@pytest.mark.parametrize("integ", [G.SE, G.GL])
def test_section_7_3_findings(integ):
    N = 1_000_000
    ad = gpu_params(dict(W.PAPER, z_adapt=XA))
    un = gpu_params(dict(W.PAPER))
    va = [_stats(ad, integ, l, N, 3)[1] for l in (3, 4, 5)]
    vu5 = _stats(un, integ, 5, N, 3)[1]
    assert all(3.0 < va[k] / va[k + 1] < 5.5 for k in range(2)), va     # beta ~ 2
    assert va[2] < vu5
    mu, _, su = _stats(un, integ, 4, N, 9)
    ma, _, sa = _stats(ad, integ, 4, N, 9)
    g = GOLDEN["adaptive_bias_ratio"]
    if integ == G.SE:
        ratio, want = abs(mu) / abs(ma), g["SE_uniform_over_adaptive"]
    else:
        ratio, want = abs(ma) / abs(mu), g["GL_adaptive_over_uniform"]
    assert want / 2 < ratio < want * 2, (mu, su, ma, sa)


def test_adaptive_is_refused_where_unsupported():
    d = dict(W.bl600(G.GL), z_adapt=30.0)
    p = gpu_params(d)
    with pytest.raises(G.MLMCError) as e:
        G.level_sums(2, 100, G.BAOAB, p, 1)
    assert e.value.code == G.EINVAL
    for call in (lambda: G.estimate_graph(1e-2, G.GL, p, 1),
                 lambda: G.path_trace(1, 4, G.GL, p, 1),
                 lambda: G.level_pdf_sums(1, 100, G.GL, gpu_params(dict(d, smooth_delta=30.0)), 1, 4)):
        with pytest.raises(G.MLMCError) as e:
            call()
        assert e.value.code == G.EINVAL
    with pytest.raises(G.MLMCError) as e:     # lambda(X_adapt) below lambda_max / 1024
        G.level_sums(2, 100, G.GL, gpu_params(dict(d, z_adapt=599.9)), 1)
    assert e.value.code == G.EINVAL


@pytest.mark.parametrize("integ", [G.SE, G.GL])
def test_adaptive_empty_single_and_ragged(integ):
    # FP64 paths, which equal the oracle's pair by pair
    d = CASES[0][1] if integ == G.SE else CASES[2][1]
    level = d["level_min"] + 1
    pg, po = gpu_params(d, G.FP64), oracle_params(d, G.FP64)
    s0 = G.level_sums(level, 0, integ, pg, 3)
    assert s0["n"] == 0 and s0["path_steps"] == 0
    for n, off in ((1, 12345), (4096 * 2 + 257, 7)):   # not a multiple of a chunk or a block
        s = G.level_sums(level, n, integ, pg, 3, path_offset=off)
        o = O.level_sums(po, integ, level, n, off, 3)
        assert s["n"] == o["n"] == n and s["path_steps"] == o["path_steps"]
        assert np.array_equal(np.array(s["sum"][1]), o["sum"][1])     # indicator counts
        assert np.allclose(s["sum"][0], o["sum"][0], rtol=1e-9, atol=1e-9 * n)


@pytest.mark.parametrize("precision", [G.FP32, G.FP64])
@pytest.mark.parametrize("case", [0, 2, 3, 4])
def test_level_sums_are_the_sums_of_the_per_pair_outputs(case, precision):
    # The level-sums kernel hands pairs out dynamically and parks their end
    # states in shared memory; the per-pair output kernel runs one pair per
    # thread.  The level sums must be the FP64 sums of the per-pair end
    # states (counts and steps exactly), and the batched launch must agree.
    integ, d, level = CASES[case]
    N = 3001
    pg = gpu_params(d, precision)
    states, flags, steps = G.level_paths(level, N, integ, pg, 23, path_offset=11, steps=True)
    gs, gf, gst = states.double().cpu().numpy(), flags.cpu().numpy(), steps.cpu().numpy()
    s = G.level_sums(level, N, integ, pg, 23, path_offset=11)
    ok = gf == 0
    assert s["n"] == ok.sum() and s["n_nonfinite"] == (~ok).sum()
    assert s["path_steps"] == int(gst.sum())
    Y = gs[ok, 0] - gs[ok, 2]
    for k, v in enumerate([Y.sum(), (Y * Y).sum(), gs[ok, 0].sum(), (gs[ok, 0] ** 2).sum(),
                           gs[ok, 2].sum(), (gs[ok, 2] ** 2).sum()]):
        assert s["sum"][0][k] == pytest.approx(v, rel=1e-12, abs=1e-9), k
    b = G.multilevel_sums([(level, 11, N)], integ, pg, 23)[0]
    assert b["n"] == s["n"] and b["path_steps"] == s["path_steps"]
    assert np.allclose(b["sum"][0], s["sum"][0], rtol=1e-11)
