"""Smoothed indicator QoI and binned density on the GPU against the oracle
(Section 5.1 and Section 6.3 of the paper).

The GPU evaluates the smoothing polynomial (solved by the library's own
reduced odd system) in the path precision; the checks are
* the sums equal float64 recomputations from the kernel's own per-path
  states, with the oracle's polynomial, to the FP32 evaluation error;
* level means agree with the oracle's to the per-path tolerance;
* the batched launch and the single-level launch agree;
* the adaptive density estimate sums to the probability mass the smoothing
  keeps inside [0, H] and matches the oracle's bin estimates.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1612_07717_gb300 import workloads as W

import paper_1612_07717_gb300 as G

from parity import gpu_params, oracle_params

pytestmark = pytest.mark.gpu

H = 600.0


def _smooth_dict(integ, r=4, delta=0.05 * H, a=0.1 * H, b=0.2 * H):
    return dict(W.bl600(integ), qoi1_mode=1, smooth_r=r, smooth_delta=delta, qoi_a=a, qoi_b=b)


def _P(coef, r, z, a, b, delta):
    def g(x):
        v = np.polyval(coef[::-1], x)
        return np.where(x < -1, 1.0, np.where(x > 1, 0.0, v))
    return g((z - b) / delta) - g((z - a) / delta)


@pytest.mark.parametrize("r", [2, 4, 8])
@pytest.mark.parametrize("integ", [G.GL, G.BAOAB, G.SE])
def test_smoothed_qoi_sums(integ, r):
    d = _smooth_dict(integ, r=r)
    level = d["level_min"] + 2
    N = 40001
    pg, po = gpu_params(d), oracle_params(d)
    s = G.level_sums(level, N, integ, pg, 3, path_offset=11)
    states, flags = G.level_paths(level, N, integ, pg, 3, path_offset=11)
    zs = states.double().cpu().numpy()
    ok = flags.cpu().numpy() == 0
    coef = O.smooth_poly(r)
    Pf = _P(coef, r, zs[ok, 0], d["qoi_a"], d["qoi_b"], d["smooth_delta"])
    Pc = _P(coef, r, zs[ok, 2], d["qoi_a"], d["qoi_b"], d["smooth_delta"])
    Y = Pf - Pc
    ref = [Y.sum(), (Y * Y).sum(), Pf.sum(), (Pf * Pf).sum(), Pc.sum(), (Pc * Pc).sum()]
    got = s["sum"][1]
    for j in range(6):
        assert abs(got[j] - ref[j]) <= 2e-6 * ok.sum(), (j, got[j], ref[j])
    o = O.level_sums(po, integ, level, N, 11, 3)
    n = o["n"]
    for j in (0, 2, 4):
        assert abs(got[j] / s["n"] - o["sum"][1][j] / n) <= 1e-4, j


def test_batched_launch_carries_the_smoothed_qoi():
    integ = G.BAOAB
    d = _smooth_dict(integ)
    pg = gpu_params(d)
    reqs = [(4, 0, 30001), (2, 0, 100000), (0, 7, 400000)]
    got = G.multilevel_sums(reqs, integ, pg, 5)
    for (l, f, n), g in zip(reqs, got):
        s = G.level_sums(l, n, integ, pg, 5, path_offset=f)
        assert g["n"] == s["n"]
        assert np.allclose(g["sum"][1], s["sum"][1], rtol=1e-11, atol=1e-9)
        assert np.allclose(g["sum"][0], s["sum"][0], rtol=1e-11)


@pytest.mark.parametrize("integ", [G.GL, G.BAOAB])
def test_pdf_level_sums_match_oracle(integ):
    k = 12
    d = dict(W.bl600(integ), smooth_r=4, smooth_delta=0.05 * H)
    level, N = 3, 20000
    pg, po = gpu_params(d), oracle_params(d)
    g = G.level_pdf_sums(level, N, integ, pg, 9, k, path_offset=3)
    o = O.level_pdf_sums(po, integ, level, N, k, offset=3, seed=9)
    assert g["n"] == o["n"] == N
    gy = np.array([g["sum"][i][0] for i in range(k)])
    oy = o["sum"][:, 0]
    assert np.all(np.abs(gy - oy) / N <= 1e-4), (gy / N, oy / N)
    # bins sum to sum_path (G_k - G_0) for fine minus coarse: telescoping
    states, flags = G.level_paths(level, N, integ, pg, 9, path_offset=3)
    zs = states.double().cpu().numpy()
    coef = O.smooth_poly(4)
    tele = lambda z: _P(coef, 4, z, 0.0, H, 0.05 * H)
    assert abs(gy.sum() - (tele(zs[:, 0]) - tele(zs[:, 2])).sum()) <= 2e-6 * N


def test_pdf_estimate_is_a_density():
    k = 10
    d = dict(W.bl600(G.BAOAB, L_max=10, n_init=5000), smooth_r=4, smooth_delta=0.05 * H)
    pg = gpu_params(d)
    eps = 2e-3
    r = G.estimate_pdf(eps, G.BAOAB, pg, 1, k)
    assert r["converged"] == 1
    pdf = np.array(r["pdf"])
    assert np.all(pdf > -3 * eps)
    # the bins sum to E[g((z - H)/delta) - g(z/delta)]: 1 away from the walls,
    # between 1/2 and 1 within delta of a wall
    assert 0.5 < pdf.sum() < 1.0 + 3 * eps
    assert math.sqrt(r["est_variance"][0]) <= eps / math.sqrt(2) * 1.05
    # the release at 0.1 H with T = 600 s keeps most particles in the lower half
    assert pdf[:5].sum() > pdf[5:].sum()
