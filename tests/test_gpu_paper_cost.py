"""Cost against tolerance in the paper's scenario for all three integrators
(Section 6.1, Fig. CostRatesPosition), on the GPU.

* MLMC cost grows like eps^-2 and plain Monte Carlo at the same finest
  timestep like eps^-3, for SE, GL and BAOAB;
* MLMC costs depend little on the integrator;
* plain Monte Carlo with the splitting methods is much cheaper than with SE
  (the paper: GL about 5x, BAOAB more than 20x), because their bias at a
  given h is 13x and 52x smaller;
* MLMC beats plain Monte Carlo at the tightest tolerance;
* the binned density's cost table of Section 6.3 (release heights 0.05,
  0.1, 0.2), in path-steps.
"""
import numpy as np
import pytest

import paper_1612_07717_gb300 as G
from paper_1612_07717_gb300 import sweeps

pytestmark = pytest.mark.gpu

EPS = [4e-4, 2e-4, 1e-4, 5e-5]


@pytest.fixture(scope="module")
def sweep():
    return {r["integrator"] + "/%g" % r["eps"]: r
            for r in sweeps.paper_cost_sweep(EPS, (G.SE, G.GL, G.BAOAB))}


@pytest.mark.parametrize("name", ["SE", "GL", "BAOAB"])
def test_cost_rates(sweep, name):
    rows = [sweep["%s/%g" % (name, e)] for e in EPS]
    assert all(r["mlmc"]["converged"] == 1 for r in rows)
    m = [r["mlmc"]["path_steps"] for r in rows]
    s = [r["stmc"]["path_steps"] for r in rows]
    sl_m = np.polyfit(np.log(EPS), np.log(m), 1)[0]
    sl_s = np.polyfit(np.log(EPS), np.log(s), 1)[0]
    # eps^-2 asymptotically; over this range the n_init floor of the coarse
    # levels and the whole-level steps of L flatten the fit a little
    assert -2.7 < sl_m < -1.4, (sl_m, m)
    assert -3.8 < sl_s < -2.3, (sl_s, s)
    assert m[-1] < s[-1]
    # both estimates land on the paper's E[X_T] = 0.1301 +- 4e-4
    for r in rows:
        for k in ("mlmc", "stmc"):
            assert abs(r[k]["estimate"] - 0.1301) < 4e-4 + 3 * r["eps"], (k, r)


def test_integrator_comparison(sweep):
    e = EPS[-1]
    m = {n: sweep["%s/%g" % (n, e)]["mlmc"]["path_steps"] for n in ("SE", "GL", "BAOAB")}
    s = {n: sweep["%s/%g" % (n, e)]["stmc"]["path_steps"] for n in ("SE", "GL", "BAOAB")}
    assert max(m.values()) / min(m.values()) < 4, m
    assert s["SE"] / s["GL"] > 2, s
    assert s["SE"] / s["BAOAB"] > 8, s
    L = {n: sweep["%s/%g" % (n, e)]["mlmc"]["L"] for n in ("SE", "GL", "BAOAB")}
    assert L["SE"] > L["GL"] >= L["BAOAB"], L


@pytest.fixture(scope="module")
def pdf_table():
    return {(r["release"], r["integrator"]): r for r in sweeps.pdf_release_table()}


def test_pdf_release_table_of_section_6_3(pdf_table):
    """The 20-bin density to RMSE 4e-3 on rho (Section 6.3's table): plain
    Monte Carlo with SE grows steeply as the release height falls while GL
    and BAOAB barely move; MLMC-SE beats StMC-SE everywhere and gets cheaper
    with height; StMC-BAOAB is the cheapest at 0.05 and MLMC-SE at 0.2."""
    st = {k: r["stmc"]["path_steps"] for k, r in pdf_table.items()}
    ml = {k: r["mlmc"]["path_steps"] for k, r in pdf_table.items()}
    assert all(r["mlmc"]["converged"] == 1 for r in pdf_table.values())
    assert st[(0.05, "SE")] > 3 * st[(0.2, "SE")]
    for name in ("GL", "BAOAB"):
        v = [st[(x, name)] for x in (0.05, 0.1, 0.2)]
        assert max(v) < 1.6 * min(v), (name, v)
    assert st[(0.05, "SE")] > 4 * st[(0.05, "GL")]
    assert st[(0.05, "SE")] > 10 * st[(0.05, "BAOAB")]
    for x in (0.05, 0.1, 0.2):
        assert ml[(x, "SE")] * 5 < st[(x, "SE")], x
    assert ml[(0.05, "SE")] > 1.3 * ml[(0.1, "SE")]
    assert ml[(0.1, "SE")] > 1.3 * ml[(0.2, "SE")]
    everything = lambda x: {**{("stmc", n): st[(x, n)] for n in ("SE", "GL", "BAOAB")},
                            **{("mlmc", n): ml[(x, n)] for n in ("SE", "GL", "BAOAB")}}
    low = everything(0.05)
    assert min(low, key=low.get) == ("stmc", "BAOAB"), low
    high = everything(0.2)
    assert high[("mlmc", "SE")] <= 1.2 * high[("stmc", "BAOAB")], high
    # the bins hold the probability mass that the smoothing keeps inside [0, H]
    for r in pdf_table.values():
        assert 0.9 < r["mlmc"]["mass"] <= 1.0 + 1e-3
