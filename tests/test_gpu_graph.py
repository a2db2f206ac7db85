"""The adaptive MLMC loop captured as one CUDA graph (GPU): its result
equals the host-driven loop's up to the FP64 rounding of the level sums, and
relaunching the instantiated graph reproduces it bit for bit."""
import math

import pytest

import paper_1612_07717_gb300 as G
from paper_1612_07717_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [G.FP64, G.FP32])
@pytest.mark.parametrize("integ", [G.GL, G.BAOAB, G.SE])
def test_graph_loop_matches_host_loop(integ, precision):
    d = W.bl600(integ, L_max=9, n_init=2000)
    p = G.make_params(d, precision=precision)
    eps = 600 * 2.0 ** -8
    h = G.estimate(eps, integ, p, 5)
    g = G.estimate_graph(eps, integ, p, 5)
    assert g["status"] == h["status"]
    assert g["L"] == h["L"] and g["converged"] == h["converged"]
    for a, b in zip(g["N"], h["N"]):
        assert abs(a - b) <= 1
    for q in range(2):
        assert g["estimate"][q] == pytest.approx(h["estimate"][q], rel=1e-9, abs=1e-9)
    assert g["total_path_steps"] == pytest.approx(h["total_path_steps"], rel=1e-6)
    se = math.sqrt(g["est_variance"][0])
    assert se <= eps / math.sqrt(2) * 1.05


def test_graph_relaunch_is_bitwise_reproducible():
    p = G.make_params(W.bl600(G.BAOAB, L_max=10, n_init=5000))
    ge = G.GraphEstimator(600 * 2.0 ** -9, G.BAOAB, p, 11)
    ge.launch()
    a = ge.result()
    ge.launch()
    b = ge.result()
    ge.close()
    for k in ("estimate", "est_variance", "N", "V", "mean_y", "L", "total_path_steps"):
        assert a[k] == b[k], k
    assert a["converged"] == 1


def test_watchdog_ends_the_device_loop_and_leaves_the_device_usable():
    # A tolerance that needs several passes, with the loop's pass limit set to
    # 2: the update kernel ends the loop and the result reports MLMC_ETIMEOUT
    # (no spin, no trap); the next graph on the same workspace runs normally.
    p = G.make_params(W.bl600(G.BAOAB, L_max=10, n_init=2000))
    eps = 600 * 2.0 ** -9
    ws = G.Workspace(p)
    ge = G.GraphEstimator(eps, G.BAOAB, p, 11, workspace=ws, max_passes=2)
    ge.launch()
    with pytest.raises(G.MLMCError) as e:
        ge.result()
    assert e.value.code == G.ETIMEOUT
    ge.close()
    with pytest.raises(G.MLMCError) as e:
        G.GraphEstimator(eps, G.BAOAB, p, 11, workspace=ws, max_passes=4 * 32 + 1)
    assert e.value.code == G.EINVAL
    r = G.estimate_graph(eps, G.BAOAB, p, 11, workspace=ws)
    assert r["status"] == G.OK and r["converged"] == 1
    ref = G.estimate(eps, G.BAOAB, p, 11)
    assert r["L"] == ref["L"]
