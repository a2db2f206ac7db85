"""Statistical and structural pins of the oracle's MLMC estimator (CPU only).

* telescoping identity: the coarse path of level l has the law of the fine
  path of level l-1 (Eq. telescoping_sum needs it);
* well-mixed invariance of the model (Section 2);
* variance decay rates: beta ~ 2 with the reflection-aware coupling, much
  less with the naive coupling (Section 4.1), beta ~ 1 for the indicator;
* the paper's printed values in its Section 6 scenario;
* determinism: thread-count independence and path_offset composability;
* the adaptive driver against Giles' Eq. 12 and its bias test.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1612_07717_gb300 import workloads as W

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _mean_se(s, q, which):
    """mean and standard error of Y (which=0), P_f (2) or P_c (4)."""
    n = s["n"]
    m1, m2 = s["sum"][q][which], s["sum"][q][which + 1]
    mean = m1 / n
    var = max(m2 / n - mean * mean, 0.0) * n / (n - 1)
    return mean, math.sqrt(var / n)


@pytest.mark.parametrize("integ,level", [(O.SE, 7), (O.GL, 3), (O.BAOAB, 3)])
def test_telescoping_coarse_law_equals_previous_fine_law(integ, level):
    p = O.make_params(W.bl600(integ))
    N = 60000 if integ != O.SE else 20000
    hi = O.level_sums(p, integ, level, N, 0, 21)
    lo = O.level_sums(p, integ, level - 1, N, 0, 22)
    for q in range(2):
        mc, sc = _mean_se(hi, q, 4)
        mf, sf = _mean_se(lo, q, 2)
        assert abs(mc - mf) < 4 * math.hypot(sc, sf), (q, mc, mf)
        # and E[Y] = E[P_f] - E[P_c] per level (sums are consistent)
        my, _ = _mean_se(hi, q, 0)
        mfh, _ = _mean_se(hi, q, 2)
        assert my == pytest.approx(mfh - mc, abs=1e-9 * max(1.0, abs(mfh)))


def test_well_mixed_state_is_preserved():
    # z ~ U(0, H), w ~ N(0, sigma_w(z)^2) must stay so (the well-mixed
    # condition, Section 2); BAOAB with 512 steps over 600 s.
    p = O.make_params(W.well_mixed(M0=512))
    N = 30000
    zs, bad = O.paths(p, O.BAOAB, 0, N, 0, 31)
    assert bad.sum() == 0
    z, w = zs[:, 0], zs[:, 1]
    H = p.H
    nb = 10
    counts, edges = np.histogram(z, bins=nb, range=(0, H))
    expected = N / nb
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert chi2 < 35.0                      # 9 dof, p ~ 1e-4
    for b in range(1, nb - 1):
        sel = (z >= edges[b]) & (z < edges[b + 1])
        zz = z[sel]
        s2 = np.array([O.coefficients(p, x)[1] for x in zz])
        ratio = np.mean(w[sel] ** 2 / s2)
        assert abs(ratio - 1.0) < 0.08, (b, ratio)


def _fit_beta(p, integ, levels, N, q=0, seed=41):
    V = []
    for l in levels:
        s = O.level_sums(p, integ, l, N, 0, seed)
        n = s["n"]
        m1, m2 = s["sum"][q][0], s["sum"][q][1]
        V.append((m2 - m1 * m1 / n) / (n - 1))
    slope = -np.polyfit(levels, np.log2(V), 1)[0]
    return slope, V


@pytest.mark.parametrize("integ", [O.GL, O.BAOAB, O.SE])
def test_variance_decay_is_quadratic_with_reflection_coupling(integ):
    p = O.make_params(W.PAPER)
    beta, V = _fit_beta(p, integ, [2, 3, 4, 5], 12000)
    assert 1.5 < beta < 2.7, (beta, V)


def test_naive_coupling_loses_variance_decay():
    p = O.make_params(W.PAPER, coupling=1)
    beta, V = _fit_beta(p, O.GL, [2, 3, 4, 5], 12000)
    assert beta < 1.2, (beta, V)
    pc = O.make_params(W.PAPER)
    _, Vc = _fit_beta(pc, O.GL, [5], 12000)
    assert V[-1] > 5 * Vc[0]


def test_indicator_variance_decays_linearly():
    p = O.make_params(W.PAPER, qoi_threshold=0.1555)
    beta, V = _fit_beta(p, O.GL, [2, 3, 4, 5, 6], 20000, q=1)
    assert 0.5 < beta < 1.5, (beta, V)


@pytest.mark.slow
def test_paper_mean_position_and_interval_probability():
    g = GOLDEN
    a, b = g["interval_probability"]["a"], g["interval_probability"]["b"]
    N = 300000
    pa = O.make_params(W.PAPER, M0=160, qoi_threshold=a)
    pb = O.make_params(W.PAPER, M0=160, qoi_threshold=b)
    sa = O.level_sums(pa, O.BAOAB, 0, N, 0, 51)
    sb = O.level_sums(pb, O.BAOAB, 0, N, 0, 51)
    mx, sx = _mean_se(sb, 0, 2)
    assert abs(mx - g["mean_position"]["value"]) < g["mean_position"]["tolerance"] + 3 * sx
    pint = (sb["sum"][1][2] - sa["sum"][1][2]) / N
    sd = math.sqrt(pint * (1 - pint) / N)
    ref = g["interval_probability"]["BAOAB"]
    assert abs(pint - ref) < g["interval_probability"]["bias_tolerance"] + 3 * sd


def test_bias_ratio_between_integrators_is_paper_like():
    # E[Y_l] = E[P_l - P_{l-1}] estimates the first-order bias at h_l, with
    # a small variance thanks to the coupling (Section 6.1 bias plot).
    p = O.make_params(W.PAPER)
    N = 40000
    means = {}
    for integ in (O.SE, O.GL):
        s = O.level_sums(p, integ, 2, N, 0, 61)
        m, se = _mean_se(s, 0, 0)
        means[integ] = (m, se)
    ratio = means[O.SE][0] / means[O.GL][0]
    assert 8.0 < abs(ratio) < 30.0, (ratio, means)     # paper: about 13


def test_thread_count_and_offset_independence():
    p = O.make_params(W.bl600(O.GL))
    s1 = O.level_sums(p, O.GL, 2, 5000, 0, 7, threads=1)
    s8 = O.level_sums(p, O.GL, 2, 5000, 0, 7, threads=8)
    assert np.array_equal(s1["sum"], s8["sum"])
    a = O.level_sums(p, O.GL, 2, 2048, 0, 7, threads=4)
    b = O.level_sums(p, O.GL, 2, 5000 - 2048, 2048, 7, threads=4)
    assert np.allclose(a["sum"] + b["sum"], s1["sum"], rtol=1e-13, atol=1e-9)
    assert a["n"] + b["n"] == s1["n"]


def test_adaptive_driver_follows_giles_rules():
    p = O.make_params(W.bl600(O.GL, L_max=8, n_init=1000))
    eps = p.H * 2.0 ** -9
    r = O.estimate(p, O.GL, eps, seed=3)
    lm = p.level_min
    L = r["L"]
    assert r["converged"] == 1
    assert L >= lm + 2
    # variance part of the MSE within eps^2 / 2 (Giles Eq. 12 makes it so,
    # up to the ceil and the variance estimates)
    assert r["est_variance"][0] <= 0.5 * eps ** 2 * 1.05
    # bias test of Giles Eq. 11 with M = 2
    yL = abs(r["mean_y"][-1])
    yL1 = abs(r["mean_y"][-2])
    assert max(yL1 / 2, yL) < eps / math.sqrt(2)
    # N_l decreasing with l, as the cost grows and V_l falls
    N = r["N"]
    assert all(N[j] >= N[j + 1] for j in range(len(N) - 1))
    # N_l proportional to sqrt(V_l / C_l): check the rule directly for the
    # levels whose N exceeds n_init
    C = [(p.M0 << l) * (1.5 if l > lm else 1.0) for l in range(lm, L + 1)]
    tot = sum(math.sqrt(v * c) for v, c in zip(r["V"], C))
    for j, (v, c) in enumerate(zip(r["V"], C)):
        nopt = 2 / eps ** 2 * math.sqrt(v / c) * tot
        if N[j] > p.n_init * 1.5:
            assert N[j] == pytest.approx(nopt, rel=0.35)


def test_n_l_ratios_resemble_paper_table():
    # Appendix C: SE, mean position, M0 = 40: N_l / N_{l+1} is 8.0 and 4.4
    # for the first two ratios, then about 3 (sqrt(V_l / C_l) falls by
    # 2^{(beta + gamma)/2} ~ 2.8 per level).  The ratios do not depend on eps.
    p = O.make_params(W.PAPER, L_max=8, n_init=4000)
    levels = list(range(0, 6))
    V, C = [], []
    for l in levels:
        s = O.level_sums(p, O.SE, l, 8000 if l < 3 else 3000, 0, 71)
        n = s["n"]
        V.append((s["sum"][0][1] - s["sum"][0][0] ** 2 / n) / (n - 1))
        M = p.M0 << l
        C.append(M if l == 0 else 1.5 * M)
    nl = [math.sqrt(v / c) for v, c in zip(V, C)]
    ratios = [nl[j] / nl[j + 1] for j in range(len(nl) - 1)]
    paper = GOLDEN["N_l_SE_mean_position"]["N"]
    pr = [paper[j] / paper[j + 1] for j in range(len(paper) - 1)]
    assert ratios[0] > 4.0 and pr[0] > 4.0
    for r in ratios[2:]:
        assert 1.8 < r < 4.5, ratios
