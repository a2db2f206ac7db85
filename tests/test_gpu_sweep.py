"""Scenario sweeps on the GPU.

* Integrator and precision sweep over (u*, z0 / H, T): FP32 paths with FP64
  sums agree with all-FP64 paths within the estimators' combined error.
* Well-mixed state over 1e8 paths: the height histogram stays flat and the
  velocity variance stays sigma_w^2, up to a discretisation error that falls
  as the step shrinks (Section 2, the well-mixed condition).
* Cost against tolerance in the paper's scenario (Section 6.1): MLMC cost
  grows like eps^-2, plain Monte Carlo at the matching step like eps^-3.
"""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1612_07717_gb300 import workloads as W

import paper_1612_07717_gb300 as G

pytestmark = pytest.mark.gpu


def _scenario(integ, u_star, z0_frac, T):
    H = 0.3 * u_star / 1e-4
    d = W.bl600(integ, u_star=u_star, H=H, z0=z0_frac * H, T=T, qoi_threshold=0.1 * H,
                L_max=12, n_init=4000)
    p = G.make_params(d)
    d["level_min"] = G.stable_level_min(p, integ)
    return d, H


@pytest.mark.parametrize("integ", [G.SE, G.GL, G.BAOAB])
@pytest.mark.parametrize("u_star,z0_frac,T", [(0.1, 0.01, 1800.0), (0.4, 0.5, 300.0),
                                             (0.2, 0.1, 600.0)])
def test_fp32_paths_agree_with_fp64_paths(integ, u_star, z0_frac, T):
    d, H = _scenario(integ, u_star, z0_frac, T)
    eps = H * 2.0 ** -8
    r32 = G.estimate_graph(eps, integ, G.make_params(d, precision=G.FP32), 17)
    r64 = G.estimate_graph(eps, integ, G.make_params(d, precision=G.FP64), 17)
    assert r32["converged"] == 1 and r64["converged"] == 1
    se = math.sqrt(r32["est_variance"][0] + r64["est_variance"][0])
    assert abs(r32["estimate"][0] - r64["estimate"][0]) <= 3 * se + 1e-4 * H


def _well_mixed_deviation(M0, N=100_000_000, bins=64):
    d = W.well_mixed(M0=M0)
    p = G.make_params(d)
    H = d["H"]
    states, flags = G.level_paths(0, N, G.BAOAB, p, 2, path_offset=0)
    assert int(flags.sum()) == 0
    z = states[:, 0]
    w = states[:, 1]
    counts = torch.histc(z, bins=bins, min=0.0, max=H).double().cpu().numpy()
    idx = torch.clamp((z / H * bins).long(), 0, bins - 1)
    w2 = torch.zeros(bins, dtype=torch.float64, device=z.device)
    w2.index_add_(0, idx, (w.double() ** 2))
    w2 = w2.cpu().numpy() / np.maximum(counts, 1)
    po = O.make_params(d)
    centres = (np.arange(bins) + 0.5) * H / bins
    s2 = np.array([O.coefficients(po, c)[1] for c in centres])
    inner = slice(2, bins - 2)
    dens = counts / (N / bins)
    return np.abs(dens[inner] - 1).max(), np.abs(w2[inner] / s2[inner] - 1).max(), dens


def test_well_mixed_state_over_1e8_paths():
    dev512, var512, dens = _well_mixed_deviation(512)
    dev2048, var2048, _ = _well_mixed_deviation(2048)
    assert dev512 < 0.03 and var512 < 0.05, (dev512, var512)
    assert dev2048 < 0.015 and var2048 < 0.03, (dev2048, var2048)
    assert dev2048 < dev512                  # the deviation falls with the step
    assert abs(dens.mean() - 1.0) < 1e-3     # nothing leaves [0, H]


def test_cost_scaling_with_tolerance_in_paper_scenario():
    d = dict(W.PAPER, L_max=12, n_init=2000)
    p = G.make_params(d)
    # tight enough that N_l, not the n_init floor, sets the cost
    eps_list = [8e-4, 4e-4, 2e-4, 1e-4]
    mlmc, stmc = [], []
    for eps in eps_list:
        r = G.estimate_graph(eps, G.GL, p, 23)
        assert r["converged"] == 1
        mlmc.append(r["total_path_steps"])
        # plain Monte Carlo at the finest MLMC step: N = 2 V / eps^2 paths
        s = G.stmc_estimate(eps, r["L"], G.GL, G.make_params(d, level_min=r["L"]), 29,
                            n_pilot=4000)
        stmc.append(s["total_path_steps"])
    sl_m = np.polyfit(np.log(eps_list), np.log(mlmc), 1)[0]
    sl_s = np.polyfit(np.log(eps_list), np.log(stmc), 1)[0]
    assert -2.6 < sl_m < -1.6, (sl_m, mlmc)
    assert -3.6 < sl_s < -2.4, (sl_s, stmc)
    assert mlmc[-1] < stmc[-1]               # MLMC wins at the tightest tolerance
