"""RMSE of the MLMC estimator (GPU) against the FP64 oracle: with FP32 BAOAB
and GL paths the adaptive estimate of E[z(T)] (the loop as one CUDA graph)
reaches RMSE <= eps for eps = 1e-3 H (Eq. MLMCerror: bias^2 + sum V_l / N_l
<= eps^2), measured over 32 independent seeds against a reference the FP64
CPU oracle computes to eps / 8 with its own, independent samples (seed 999,
the FP64 uniform map).  A bias shared by every GPU estimate would show here;
it would cancel against a GPU-computed reference.  ``pytest -s`` prints
RMSE / eps per integrator."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1612_07717_gb300 import workloads as W

import paper_1612_07717_gb300 as G

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("integ", [G.BAOAB, G.GL])
def test_rmse_within_eps_against_the_oracle(integ):
    H = 600.0
    eps = 1e-3 * H
    d = W.bl600(integ, L_max=14, n_init=10000)
    po = O.make_params(d, uniform_map=O.U32)
    ref = O.estimate(po, integ, eps / 8, seed=999)
    assert ref["converged"] == 1
    p = G.make_params(d)
    est = []
    for seed in range(100, 132):
        r = G.estimate_graph(eps, integ, p, seed)
        assert r["converged"] == 1
        est.append(r["estimate"][0])
    est = np.array(est)
    rmse = math.sqrt(np.mean((est - ref["estimate"][0]) ** 2))
    print("\nRMSE / eps (%s, 32 seeds, oracle reference %.5f m at eps/8): %.3f; "
          "mean offset / eps %.3f" % ({G.BAOAB: "BAOAB", G.GL: "GL"}[integ],
                                      ref["estimate"][0], rmse / eps,
                                      (est.mean() - ref["estimate"][0]) / eps))
    # 32 samples: the RMSE estimate itself is uncertain by about 1/sqrt(64)
    assert rmse <= 1.3 * eps, (rmse, eps, ref["estimate"][0], est.mean())
