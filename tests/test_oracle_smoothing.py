"""Pins of the oracle's smoothed indicator and binned density (CPU only),
Section 5.1 and Section 6.3 of the paper.

* p_r is symmetric: p(s) + p(-s) = 1 (the step function's defining
  conditions are invariant under s -> -s, 1 - p);
* g_r turns the step function's expectation into a smooth one with weak
  error O(delta^{r+1}) (Section 5.2): checked against the normal CDF by
  quadrature, with the convergence rate in delta;
* the smoothed interval probability of the paper's scenario matches its
  table of estimates for r = 4, delta = 0.1;
* the binned density telescopes: the bins' smoothed QoIs sum to
  g((z - H)/delta) - g(z/delta), and a bin equals the scalar smoothed QoI of
  the same interval.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, stats

from oracle import oracle as O
from paper_1612_07717_gb300 import workloads as W

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.mark.parametrize("r", [0, 1, 2, 4, 6, 8])
def test_polynomial_symmetry_and_end_values(r):
    c = O.smooth_poly(r)
    for s in np.linspace(-1, 1, 21):
        assert O.g(r, c, s) + O.g(r, c, -s) == pytest.approx(1.0, abs=1e-10)
    assert O.g(r, c, -1.0) == pytest.approx(1.0, abs=1e-12)
    assert O.g(r, c, 1.0) == pytest.approx(0.0, abs=1e-12)
    assert O.g(r, c, -1.5) == 1.0 and O.g(r, c, 1.5) == 0.0


def test_low_orders_are_the_linear_ramp():
    # r = 0 and r = 1 both give p(s) = (1 - s) / 2 (the r = 1 moment
    # condition holds for the ramp already)
    for r in (0, 1):
        c = O.smooth_poly(r)
        for s in np.linspace(-1, 1, 9):
            assert O.g(r, c, s) == pytest.approx((1 - s) / 2, abs=1e-12)


@pytest.mark.parametrize("r", [2, 4])
def test_weak_error_is_order_delta_r_plus_1(r):
    # E[g_r((X - s)/delta)] for X ~ N(0, 1) against P[X <= s] = Phi(s)
    c = O.smooth_poly(r)
    s0 = 0.3

    def err(delta):
        f = lambda x: O.g(r, c, (x - s0) / delta) * stats.norm.pdf(x)
        val, _ = integrate.quad(f, s0 - delta, s0 + delta, epsabs=1e-14, epsrel=1e-13)
        val += stats.norm.cdf(s0 - delta)
        return abs(val - stats.norm.cdf(s0))

    e = [err(d) for d in (0.4, 0.2, 0.1)]
    rates = [math.log2(e[k] / e[k + 1]) for k in range(2)]
    assert min(rates) > r + 1 - 0.3, (e, rates)


@pytest.mark.slow
def test_smoothed_interval_probability_matches_paper_table():
    g = GOLDEN["interval_probability"]
    a, b = g["a"], g["b"]
    N = 300000
    p = O.make_params(W.PAPER, M0=160, qoi1_mode=1, qoi_a=a, qoi_b=b, smooth_delta=0.1,
                      smooth_r=4)
    s = O.level_sums(p, O.BAOAB, 0, N, 0, 51)
    est = s["sum"][1][2] / s["n"]
    sd = math.sqrt(max(s["sum"][1][3] / s["n"] - est ** 2, 0.0) / s["n"])
    # paper, r = 4, delta = 0.1: GL 0.16678, SE 0.16705, BAOAB 0.16687
    assert abs(est - 0.16687) < g["bias_tolerance"] + 3 * sd, (est, sd)


def test_binned_density_telescopes_and_matches_scalar_qoi():
    H = 600.0
    k = 12
    delta = 0.05 * H
    d = dict(W.bl600(O.GL), smooth_delta=delta, smooth_r=4)
    p = O.make_params(d)
    level, N = 3, 3000
    pdf = O.level_pdf_sums(p, O.GL, level, N, k, offset=0, seed=5)
    zs, bad = O.paths(p, O.GL, level, N, 0, 5)
    c = O.smooth_poly(4)
    G = lambda z: O.g(4, c, (z - H) / delta) - O.g(4, c, z / delta)
    tele_f = sum(G(z) for z in zs[:, 0])
    tele_c = sum(G(z) for z in zs[:, 2])
    assert pdf["sum"][:, 2].sum() == pytest.approx(tele_f, rel=1e-12)
    assert pdf["sum"][:, 4].sum() == pytest.approx(tele_c, rel=1e-12)
    i = 3
    ps = O.make_params(d, qoi1_mode=1, qoi_a=i * H / k, qoi_b=(i + 1) * H / k)
    sc = O.level_sums(ps, O.GL, level, N, 0, 5)
    assert np.allclose(sc["sum"][1], pdf["sum"][i], rtol=1e-12, atol=1e-12)
