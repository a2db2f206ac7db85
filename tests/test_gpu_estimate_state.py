"""Checkpoint and resume of the host-driven estimator (GPU): the pass-by-pass
form gives mlmc_estimate's result bit for bit, and a run stopped after some
passes, written to JSON and resumed in a new object, gives it too."""
import json

import pytest

from paper_1612_07717_gb300 import workloads as W

import paper_1612_07717_gb300 as G

pytestmark = pytest.mark.gpu

KEYS = ("estimate", "est_variance", "N", "V", "mean_y", "L", "converged", "total_path_steps",
        "n_nonfinite")


def _same(a, b):
    for k in KEYS:
        assert a[k] == b[k], k


@pytest.mark.parametrize("integ", [G.GL, G.BAOAB])
def test_passes_give_the_estimate(integ):
    p = G.make_params(W.bl600(integ, n_init=4000, L_max=10))
    eps = 600 * 2.0 ** -9
    ref = G.estimate(eps, integ, p, 5)
    e = G.Estimation(eps, integ, p, 5)
    n = 0
    while not e.step():
        n += 1
    _same(e.result(), ref)
    assert e.state.passes == n + 1 == 2 * (ref["L"] - p.level_min + 1)


def test_resume_from_json_gives_the_uninterrupted_result(tmp_path):
    integ = G.BAOAB
    p = G.make_params(W.bl600(integ, n_init=4000, L_max=10))
    eps = 600 * 2.0 ** -10
    ref = G.estimate(eps, integ, p, 9)
    first = G.Estimation(eps, integ, p, 9)
    for _ in range(3):
        assert not first.step()
    path = str(tmp_path / "state.json")
    with open(path, "w") as f:
        json.dump(first.state_dict(), f)
    del first                                   # the "crash"
    again = G.Estimation(eps, integ, p, 9)      # a fresh process would do the same
    r = again.run(checkpoint=path)              # resumes from the file, rewrites it
    _same(r, ref)
    with open(path) as f:
        assert json.load(f)["phase"] == 2


def test_measured_rates_of_an_estimate():
    # the coupled splitting scheme's variance decays about like h^2 (Section 6.1)
    p = G.make_params(W.PAPER, precision=G.FP32)
    r = G.estimate(5e-5, G.BAOAB, p, 3)
    assert r["L"] - p.level_min >= 3
    rt = G.rates(r, p.level_min)
    assert 1.5 < rt["beta"] < 3.0, rt
