"""Cost against tolerance in the paper's scenario (Section 6.1, Fig.
CostRatesPosition; Section 7.3 for adaptive timesteps; Section 6.3's table of
the binned density's cost for three release heights).

For each RMSE tolerance eps on E[X_T] and each integrator:

* MLMC: the adaptive estimator (``estimate_graph``, or the host-driven
  ``estimate`` for adaptive timesteps); cost = integrator steps taken;
* StMC: plain Monte Carlo at the finest timestep the MLMC hierarchy needed
  for the same eps (so both have the same bias), N = 2 Var / eps^2 paths
  (``stmc_estimate``).

Both use FP32 paths with FP64 sums, so the step counts compare the two
algorithms on equal terms.

Run on a GPU: ``python -m paper_1612_07717_gb300.sweeps [out.json]``.
``python -m paper_1612_07717_gb300.sweeps time_to_eps`` times MLMC against
plain FP64 Monte Carlo in the 600 m layer for eps = H 2^-9 .. H 2^-13;
``python -m paper_1612_07717_gb300.sweeps scenarios`` runs the integrator and
precision sweep over (u*, z0 / H, T).
"""
import json
import math
import sys
import time

from . import (BAOAB, FP32, FP64, GL, SE, Workspace, estimate, estimate_graph, estimate_pdf,
               level_pdf_sums, make_params, stmc_estimate)
from . import workloads as W

NAMES = {SE: "SE", GL: "GL", BAOAB: "BAOAB"}
EPS = (1e-3, 5e-4, 2e-4, 1e-4, 5e-5)


def mlmc_cost(eps, integ, seed=1, z_adapt=0.0, n_init=4000, L_max=12, precision=FP32):
    d = dict(W.PAPER, n_init=n_init, L_max=L_max, z_adapt=z_adapt)
    p = make_params(d, precision=precision)
    ws = Workspace(p)
    run = estimate if z_adapt > 0 else estimate_graph
    run(eps, integ, p, seed + 1000, workspace=ws)   # warm-up: module loading, first graph
    t = time.perf_counter()
    r = run(eps, integ, p, seed, workspace=ws)
    dt = time.perf_counter() - t
    return dict(L=r["L"], converged=r["converged"], estimate=r["estimate"][0],
                rmse_stat=math.sqrt(r["est_variance"][0]), path_steps=r["total_path_steps"],
                seconds=dt, N=r["N"])


def stmc_cost(eps, integ, level, seed=2, n_pilot=4000, precision=FP32):
    p = make_params(dict(W.PAPER, level_min=level), precision=precision)
    ws = Workspace(p)
    stmc_estimate(eps, level, integ, p, seed + 1000, n_pilot=n_pilot, workspace=ws)  # warm-up
    t = time.perf_counter()
    s = stmc_estimate(eps, level, integ, p, seed, n_pilot=n_pilot, workspace=ws)
    dt = time.perf_counter() - t
    return dict(level=level, h=W.PAPER["T"] / (W.PAPER["M0"] << level), N=s["N"][0],
                estimate=s["estimate"][0], path_steps=s["total_path_steps"], seconds=dt)


def bl600_time_to_eps(eps_fracs=(2.0 ** -9, 2.0 ** -10, 2.0 ** -11, 2.0 ** -12, 2.0 ** -13),
                      seed=3, n_init=2000, n_pilot=2000):
    """Wall time to RMSE eps = H * frac on E[z(T)] in the 600 m layer: MLMC
    with FP32 GL and BAOAB paths (the adaptive loop in one CUDA graph, after
    one warm-up run) against plain Monte Carlo with FP64 symplectic-Euler
    paths at the finest level the SE hierarchy needs for the same eps."""
    import torch
    H = W.BL600["H"]
    out = []
    # load the FP64 kernels before the first timed call
    pw = make_params(W.bl600(SE), precision=FP64, level_min=8)
    stmc_estimate(H * 2.0 ** -6, 8, SE, pw, seed + 400, n_pilot=n_pilot, workspace=Workspace(pw))
    for frac in eps_fracs:
        eps = H * frac
        row = dict(eps_over_H=frac, eps_m=eps)
        for name, integ in (("gl", GL), ("baoab", BAOAB)):
            p = make_params(W.bl600(integ, L_max=14, n_init=n_init), precision=FP32)
            ws = Workspace(p)
            estimate_graph(eps, integ, p, seed + 100, workspace=ws)
            torch.cuda.synchronize()
            t = time.perf_counter()
            r = estimate_graph(eps, integ, p, seed, workspace=ws)
            row["mlmc_" + name] = dict(seconds=time.perf_counter() - t, L=r["L"],
                                       path_steps=r["total_path_steps"],
                                       estimate_m=r["estimate"][0])
        pse = make_params(W.bl600(SE, L_max=16, n_init=n_init), precision=FP32)
        level = estimate_graph(eps, SE, pse, seed + 200, workspace=Workspace(pse))["L"]
        p64 = make_params(W.bl600(SE), precision=FP64, level_min=level)
        ws64 = Workspace(p64)
        t = time.perf_counter()
        s = stmc_estimate(eps, level, SE, p64, seed + 300, n_pilot=n_pilot, workspace=ws64)
        row["stmc_fp64_se"] = dict(seconds=time.perf_counter() - t, level=level, N=s["N"][0],
                                   path_steps=s["total_path_steps"], estimate_m=s["estimate"][0])
        out.append(row)
    return out


def scenario_precision_sweep(u_stars=(0.1, 0.2, 0.4), z0_fracs=(0.01, 0.1, 0.5),
                             Ts=(300.0, 600.0, 1800.0), eps_frac=2.0 ** -8, seed=17):
    """The integrator and precision sweep of the 1-D boundary layer: for
    every (u*, z0 / H, T) with H = 0.3 u* / f and each integrator, the MLMC
    estimate of E[z(T)] to eps = H eps_frac with FP32 paths and with FP64
    paths (FP64 sums in both; the whole loop in one CUDA graph); SE starts at
    its stable level.  Returns one record per (scenario, integrator) with
    both estimates, their standard errors and |difference| / combined SE."""
    from . import stable_level_min
    out = []
    for u in u_stars:
        for zf in z0_fracs:
            for T in Ts:
                H = 0.3 * u / W.BL600["f_coriolis"]
                for integ in (SE, GL, BAOAB):
                    d = W.bl600(integ, u_star=u, H=H, z0=zf * H, T=T, qoi_threshold=0.1 * H,
                                L_max=12, n_init=4000)
                    d["level_min"] = stable_level_min(make_params(d), integ)
                    row = dict(u_star=u, z0_over_H=zf, T=T, H=H, integrator=NAMES[integ],
                               level_min=d["level_min"])
                    for name, prec in (("fp32", FP32), ("fp64", FP64)):
                        p = make_params(d, precision=prec)
                        t = time.perf_counter()
                        r = estimate_graph(H * eps_frac, integ, p, seed, workspace=Workspace(p))
                        row[name] = dict(estimate=r["estimate"][0],
                                         se=math.sqrt(r["est_variance"][0]), L=r["L"],
                                         converged=r["converged"],
                                         path_steps=r["total_path_steps"],
                                         seconds=time.perf_counter() - t)
                    row["z"] = abs(row["fp32"]["estimate"] - row["fp64"]["estimate"]) / math.sqrt(
                        row["fp32"]["se"] ** 2 + row["fp64"]["se"] ** 2)
                    out.append(row)
    return out


def paper_cost_sweep(eps_list=EPS, integrators=(SE, GL, BAOAB)):
    out = []
    for integ in integrators:
        for eps in eps_list:
            m = mlmc_cost(eps, integ)
            s = stmc_cost(eps, integ, m["L"])
            out.append(dict(integrator=NAMES[integ], eps=eps, mlmc=m, stmc=s))
    return out


def adaptive_cost_sweep(eps_list=EPS, integrators=(SE, GL), x_adapt=0.05):
    out = []
    for integ in integrators:
        for eps in eps_list:
            out.append(dict(integrator=NAMES[integ], eps=eps,
                            uniform=mlmc_cost(eps, integ),
                            adaptive=mlmc_cost(eps, integ, z_adapt=x_adapt)))
    return out


def _pdf_params(integ, x0, level_min=0):
    # Section 6.3: r = 4, delta = 0.1, M0 = 80 for SE and GL, 40 for BAOAB
    return make_params(dict(W.PAPER, z0=x0, M0=40 if integ == BAOAB else 80, smooth_r=4,
                            smooth_delta=0.1, n_init=4000, L_max=12, level_min=level_min),
                       precision=FP32)


def stmc_pdf(eps, integ, x0, level, k=20, seed=6, n_pilot=4000):
    """Plain Monte Carlo for the k-bin density at level's timestep: a pilot
    run, then N = 2 max_i Var[P_i] / eps^2 paths in total."""
    import torch
    p = _pdf_params(integ, x0, level_min=level)
    ws = Workspace(p)
    torch.cuda.synchronize()
    t = time.perf_counter()
    a = level_pdf_sums(level, n_pilot, integ, p, seed, k, workspace=ws)
    n = a["n"]
    v = max(max(s2 / n - (s1 / n) ** 2, 0.0) for s1, s2 in a["sum"])
    N = max(n_pilot, int(math.ceil(2.0 * v / eps ** 2)))
    sums = [list(x) for x in a["sum"]]
    if N > n_pilot:
        b = level_pdf_sums(level, N - n_pilot, integ, p, seed, k, path_offset=n_pilot,
                           workspace=ws)
        sums = [[x[0] + y[0], x[1] + y[1]] for x, y in zip(sums, b["sum"])]
        n += b["n"]
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    M = p.M0 << level
    return dict(level=level, N=n, path_steps=N * M, seconds=dt, pdf=[s[0] / n for s in sums])


def pdf_release_table(eps_density=4e-3, k=20, releases=(0.05, 0.1, 0.2), seed=5):
    """Section 6.3's table: cost of the 20-bin density to RMSE eps_density
    for release heights 0.05, 0.1, 0.2 -- MLMC (SE, GL, BAOAB) and plain
    Monte Carlo at the MLMC hierarchy's finest timestep.  The tolerance is on
    the density rho = P_i / (H / k); the estimators return the bins'
    probabilities P_i, so they run at eps = eps_density H / k."""
    import torch
    eps = eps_density * W.PAPER["H"] / k
    out = []
    for x0 in releases:
        for integ in (SE, GL, BAOAB):
            p = _pdf_params(integ, x0)
            ws = Workspace(p)
            estimate_pdf(eps * 2, integ, p, seed + 1, k, workspace=ws)      # warm-up
            torch.cuda.synchronize()
            t = time.perf_counter()
            r = estimate_pdf(eps, integ, p, seed, k, workspace=ws)
            dt = time.perf_counter() - t
            m = dict(L=r["L"], converged=r["converged"], N=r["N"],
                     path_steps=r["total_path_steps"], seconds=dt, mass=sum(r["pdf"]))
            s = stmc_pdf(eps, integ, x0, r["L"], k)
            out.append(dict(release=x0, integrator=NAMES[integ], mlmc=m,
                            stmc=dict(level=s["level"], N=s["N"], path_steps=s["path_steps"],
                                      seconds=s["seconds"])))
    return out


if __name__ == "__main__" and len(sys.argv) > 1 and sys.argv[1] == "scenarios":
    print(json.dumps(scenario_precision_sweep(), indent=1))
elif __name__ == "__main__" and len(sys.argv) > 1 and sys.argv[1] == "time_to_eps":
    print(json.dumps(bl600_time_to_eps(), indent=1))
elif __name__ == "__main__":
    res = dict(scenario="paper (H = 1, u* = 0.2, T = 1, X0 = 0.05, U0 = 0.1, eps_reg = 0.01, M0 = 40)",
               cost=paper_cost_sweep(), adaptive=adaptive_cost_sweep(),
               pdf=pdf_release_table())
    text = json.dumps(res, indent=1)
    if len(sys.argv) > 1:
        with open(sys.argv[1], "w") as f:
            f.write(text)
    print(text)
