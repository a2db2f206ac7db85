"""RMSE of the MLMC estimator (GPU): with FP32 BAOAB paths the adaptive
estimate of E[z(T)] reaches RMSE <= eps for eps = 1e-3 H, measured over
independent seeds against a reference computed to eps / 8."""
import math

import numpy as np
import pytest

import paper_1612_07717_gb300 as G
from paper_1612_07717_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("integ", [G.BAOAB, G.GL])
def test_rmse_within_eps(integ):
    H = 600.0
    eps = 1e-3 * H
    p = G.make_params(W.bl600(integ, L_max=14, n_init=10000))
    ref = G.estimate_graph(eps / 8, integ, p, 999)
    assert ref["converged"] == 1
    est = []
    for seed in range(100, 132):
        r = G.estimate_graph(eps, integ, p, seed)
        assert r["converged"] == 1
        est.append(r["estimate"][0])
    est = np.array(est)
    rmse = math.sqrt(np.mean((est - ref["estimate"][0]) ** 2))
    # 32 samples: the RMSE estimate itself is uncertain by about 1/sqrt(64)
    assert rmse <= 1.3 * eps, (rmse, eps, ref["estimate"][0], est.mean())
