"""Poisson-arrival driver of the query server (the serving workload).

Queries arrive as a Poisson stream; each has its own boundary layer and
tolerance drawn from seeded distributions (u* ~ U[0.1, 0.5] m/s,
H ~ U[300, 1500] m, z0/H ~ U[0.01, 0.5], T ~ U[300, 3600] s,
eps/H in {2^-6, 2^-8, 2^-10}), BAOAB paths, Philox stream = query number.
The driver submits each query at its arrival time and ticks the server
between arrivals; latency is submit-to-finish wall time.
"""
import time

import numpy as np

from . import BAOAB, FP32, Server, make_params
from . import workloads as W


def draw_queries(n, rate_hz=200.0, seed=7):
    """Arrival offsets [s] and parameter dicts of n queries."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=n)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for q in range(n):
        H = float(rng.uniform(300.0, 1500.0))
        d = dict(W.BL600, u_star=float(rng.uniform(0.1, 0.5)), H=H,
                 z0=float(rng.uniform(0.01, 0.5)) * H, T=float(rng.uniform(300.0, 3600.0)),
                 qoi_threshold=0.1 * H, stream_id=q, level_min=0, L_max=12, n_init=2000)
        eps = H * float(rng.choice([2.0 ** -6, 2.0 ** -8, 2.0 ** -10]))
        out.append((float(t[q]), d, eps))
    return out


def run(n=2000, rate_hz=200.0, seed=7, max_active=128, integrator=BAOAB, precision=FP32):
    """Serve n Poisson arrivals in real time; return latency and throughput."""
    queries = draw_queries(n, rate_hz, seed)
    srv = Server(integrator=integrator, precision=precision, max_active=max_active, seed=1)
    ids = []
    t0 = time.perf_counter()
    k = 0
    pool_peak = 0
    while k < n or srv.stats()["active"] + srv.stats()["queued"] > 0:
        now = time.perf_counter() - t0
        while k < n and queries[k][0] <= now:
            _, d, eps = queries[k]
            ids.append(srv.submit(make_params(d, precision=precision), eps))
            k += 1
        srv.tick()
        pool_peak = max(pool_peak, srv.pool()[0])
        if k < n and srv.stats()["active"] + srv.stats()["queued"] == 0:
            time.sleep(max(0.0, min(0.001, queries[k][0] - (time.perf_counter() - t0))))
    wall = time.perf_counter() - t0
    lat, steps, results = [], 0, []
    for qid in ids:
        r = srv.poll(qid)
        lat.append(r["latency_s"])
        steps += r["total_path_steps"]
        results.append(r)
    st = srv.stats()
    srv_pool = srv.pool()[1]
    srv.close()
    lat = np.array(lat)
    return dict(queries=n, rate_hz=rate_hz, wall_s=wall, throughput_qps=n / wall,
                path_steps_per_s=steps / wall, p50_ms=1e3 * float(np.percentile(lat, 50)),
                p99_ms=1e3 * float(np.percentile(lat, 99)), mean_ms=1e3 * float(lat.mean()),
                ticks=st["ticks"], max_active=max_active, pool_bytes=srv_pool,
                pool_peak_bytes=pool_peak,
                converged=int(sum(r["converged"] for r in results))), results, queries
