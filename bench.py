"""Benchmark of the MLMC dispersion hot path on GB300.

One step = one pass of the whole hot path over the batched multi-level
workload: all MLMC levels l = 0..12 of the 600 m boundary layer with N_l =
1e9 * 10^(-l/2) path pairs (1e9 on level 0 down to 1e3 on level 12), BAOAB
integrator, FP32 paths, FP64 compensated sums, in ONE persistent launch,
followed by the fixed-order per-level reduction -- about 2.85e10 path-steps.

Prints one JSON line (see the keys below).  ``--impl reference`` times the
FP64 CPU oracle on a bounded sample of the same workload instead.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

INTEGRATOR = 2          # BAOAB
LEVELS = 13
N0 = 1e9
# FP32 arithmetic per path-step of a coupled BAOAB level, counted from the
# step formulas as the kernel evaluates them (FMA = 2; add, multiply,
# reciprocal, reciprocal square root, exp2, log2, sin, cos = 1; compares,
# selects, min/max = 0).  A BAOAB step is 53 (B 5, A + fold 3, profile 11,
# O-step factors 16, O 3, A + fold 3, drift terms 7, B 5); per coupled pair
# of fine steps: 3 BAOAB steps, the coarse coupling 9 and one Box-Muller pair
# 13 -> 181 / 3 path-steps.
FLOPS_PER_PATH_STEP = 181.0 / 3.0
# ncu figures of the path kernel, valid only for the kernel sources they were
# taken with (their SHA-1, see kernel_sha1): DRAM bytes per full-size launch
# (launch list), the FMA-pipe, heavy-FMA-pipe and issue-slot activity of the
# full-size launch (one-pass metric captures) and, from the full capture of the
# 1e8-path case, the thread instructions per path-step.
TRAFFIC = {"kernel_sha1": "bbff457a9eab73fdc81666ad40f83962b3732fda", "bytes_per_launch": 0.945e6,
           "fma_pipe_active_pct": 57.2, "fmaheavy_pipe_active_pct": 61.2,
           "issue_active_pct": 72.0, "thread_inst_per_path_step": 69.8}
# The sources the persistent FP32 path kernels are compiled from.
KERNEL_SOURCES = ("include/mlmc.h", "paper_1612_07717_gb300/csrc/mlmc_internal.h",
                  "paper_1612_07717_gb300/csrc/mlmc_device.cuh",
                  "paper_1612_07717_gb300/csrc/mlmc_device_x2.cuh",
                  "paper_1612_07717_gb300/csrc/mlmc_kernels.cuh",
                  "paper_1612_07717_gb300/csrc/mlmc_reduce.cuh",
                  "paper_1612_07717_gb300/csrc/mlmc_kernels_inst.inc",
                  "paper_1612_07717_gb300/csrc/mlmc_kernels_f32.cu",
                  "paper_1612_07717_gb300/csrc/mlmc_kernels_f32_b3.cu",
                  "paper_1612_07717_gb300/csrc/mlmc_kernels_f32_b4.cu",
                  "paper_1612_07717_gb300/csrc/mlmc_kernels_f32_x2.cu",
                  "paper_1612_07717_gb300/csrc/mlmc_kernels_f32_x2b3.cu")


def kernel_sha1():
    """SHA-1 of KERNEL_SOURCES with comments and whitespace removed: it
    changes with the code the kernels are compiled from, not with their
    documentation."""
    import hashlib
    import re
    token = re.compile(r'//[^\n]*|/\*.*?\*/|"(?:\\.|[^"\\])*"|\s+', re.S)

    def code(text):
        # comments out first, then every whitespace run (comment lines included) to one space
        text = token.sub(lambda m: "" if m.group(0)[0] == "/" else m.group(0), text)
        return token.sub(lambda m: m.group(0) if m.group(0).startswith('"') else " ", text)
    h = hashlib.sha1()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, name), encoding="utf-8") as f:
            h.update(name.encode() + b"\0" + code(f.read()).encode())
    return h.hexdigest()


ORACLE_SAMPLE_SCALE = 2e-3


def workload():
    from paper_1612_07717_gb300 import workloads as W
    return W.schedule_c4(levels=LEVELS, n0=N0)


def path_steps_of(sched, M0=8):
    tot = 0
    for l, n in sched:
        M = M0 << l
        tot += n * (M + M // 2 if l > 0 else M)
    return tot


def sample_clocks(stop_file, out_file):
    cmd = ["nvidia-smi", "--query-gpu=clocks.sm,clocks.max.sm,power.draw,"
           "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
           "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
           "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-i", "0",
           "-lms", "100"]
    try:
        return subprocess.Popen(cmd, stdout=open(out_file, "w"), stderr=subprocess.DEVNULL)
    except Exception:
        return None


def parse_clocks(path):
    sm, mx, reasons = [], [], set()
    try:
        for line in open(path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
    except FileNotFoundError:
        pass
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx) if mx else None,
            "samples": len(sm), "reasons": sorted(reasons)}


def fp32_peak_probe(torch, lib_probe=None):
    """Measured FP32 FMA rate (FLOP/s) of this GPU from the library's probe kernel."""
    import ctypes as C
    import paper_1612_07717_gb300 as G
    L = G.lib()
    if not hasattr(L, "mlmc_fp32_peak_probe"):
        return None
    L.mlmc_fp32_peak_probe.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]
    buf = torch.empty(1 << 20, dtype=torch.float32, device="cuda")
    out = C.c_double()
    best = 0.0
    for _ in range(3):
        rc = L.mlmc_fp32_peak_probe(4096, C.c_void_p(buf.data_ptr()),
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream),
                                    C.byref(out))
        if rc == 0:
            best = max(best, out.value)
    return best or None


def workload_config(sched=None):
    """The workload keys both arms report."""
    sched = sched or workload()
    return {"workload": "batched-multilevel-l0-12-bl600-baoab", "levels": "0..12",
            "N_l": "1e9*10^(-l/2) (level 0: %d, level 12: %d)" % (sched[0][1], sched[-1][1]),
            "path_steps_per_step": path_steps_of(sched), "integrator": "BAOAB"}


def run_reference(args):
    """FP64 CPU oracle on a bounded sample of the same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_1612_07717_gb300 import workloads as W
    threads = os.cpu_count() or 1
    po = O.make_params(W.bl600(INTEGRATOR), uniform_map=O.U23)
    sched = [(l, max(1, int(round(n * ORACLE_SAMPLE_SCALE)))) for l, n in workload()]
    steps = path_steps_of(sched)

    def one(seed):
        t = time.perf_counter()
        for l, n in sched:
            O.level_sums(po, INTEGRATOR, l, n, 0, seed, threads=threads)
        return time.perf_counter() - t

    for w in range(args.warmup):
        one(100 + w)
    ts = [one(1 + k) for k in range(args.steps)]
    ms = 1e3 * sum(ts) / len(ts)
    value = steps / (ms / 1e3)
    sample = ("levels 0..12 of the batched BAOAB workload with N_l scaled by %g (%d path-steps "
              "per step)" % (ORACLE_SAMPLE_SCALE, steps))
    line = {
        "impl": "reference",
        "metric": "path-steps/s", "value": value, "unit": "path-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": dict(workload_config(), paths="fp64 (oracle)",
                       sample="N_l x %g per step: %d path-steps" % (ORACLE_SAMPLE_SCALE, steps)),
        "cpu_baseline": {"value": value, "unit": "path-steps/s", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "path-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def cpu_baseline_sample():
    """Oracle throughput on host cores for the cpu_baseline key (about 10 s)."""
    from oracle import oracle as O
    from paper_1612_07717_gb300 import workloads as W
    threads = os.cpu_count() or 1
    po = O.make_params(W.bl600(INTEGRATOR), uniform_map=O.U23)
    sched = [(l, max(1, int(round(n * ORACLE_SAMPLE_SCALE)))) for l, n in workload()]
    steps = path_steps_of(sched)
    t = time.perf_counter()
    for l, n in sched:
        O.level_sums(po, INTEGRATOR, l, n, 0, 1, threads=threads)
    dt = time.perf_counter() - t
    # one core, on a sixteenth of the sample
    sched1 = [(l, max(1, int(round(n * ORACLE_SAMPLE_SCALE / 16)))) for l, n in workload()]
    steps1 = path_steps_of(sched1)
    t = time.perf_counter()
    for l, n in sched1:
        O.level_sums(po, INTEGRATOR, l, n, 0, 1, threads=1)
    dt1 = time.perf_counter() - t
    return {"value": steps / dt, "unit": "path-steps/s", "cores": threads, "kind": "oracle",
            "sample": "levels 0..12 of the same workload with N_l x %g (%d path-steps, %.1f s)"
                      % (ORACLE_SAMPLE_SCALE, steps, dt),
            "single_core": {"value": steps1 / dt1, "unit": "path-steps/s", "cores": 1,
                            "sample": "N_l x %g (%d path-steps, %.1f s)"
                                      % (ORACLE_SAMPLE_SCALE / 16, steps1, dt1)}}


def _spread(ts):
    return {"median": statistics.median(ts), "min": min(ts), "max": max(ts), "repeats": len(ts)}


def time_to_eps(G, W, torch, eps_frac=2.0 ** -10, repeats=5):
    """Wall time to RMSE eps = H * eps_frac on mean z(T): MLMC with FP32
    BAOAB and GL paths (the adaptive loop as one CUDA graph; the faster one
    is compared) against plain Monte Carlo with FP64 symplectic-Euler paths
    at the timestep the SE hierarchy needs for the same eps (its finest
    level).  Each arm is timed `repeats` times after a warm-up (the same
    seed, so the same work); the median is compared and the spread reported."""
    H = W.BL600["H"]
    eps = H * eps_frac
    out = {"eps_m": eps}
    best = None
    for name, integ in (("baoab", G.BAOAB), ("gl", G.GL)):
        pb = G.make_params(W.bl600(integ, L_max=14, n_init=10000), precision=G.FP32)
        ws = G.Workspace(pb)
        ge = G.GraphEstimator(eps, integ, pb, 3, workspace=ws)
        ge.launch(); ge.result()                    # warm-up (module load, first launch)
        ts = []
        for _ in range(repeats):
            torch.cuda.synchronize()
            t = time.perf_counter()
            ge.launch()
            r = ge.result()
            ts.append(time.perf_counter() - t)
        ge.close()
        sp = _spread(ts)
        out["mlmc_fp32_%s_graph" % name] = {
            "seconds": sp["median"], "seconds_spread": sp, "L": r["L"],
            "estimate_m": r["estimate"][0], "rmse_stat_m": math.sqrt(r["est_variance"][0]),
            "path_steps": r["total_path_steps"], "N": r["N"], "converged": r["converged"]}
        if best is None or sp["median"] < best[1]:
            best = (name, sp["median"])
    out["mlmc_best"] = best[0]
    dt = best[1]
    # the SE hierarchy's finest level for this eps sets the plain-MC timestep
    pse = G.make_params(W.bl600(G.SE, L_max=16, n_init=10000), precision=G.FP32)
    rse = G.estimate_graph(eps, G.SE, pse, 5, workspace=ws)
    level = rse["L"]
    p64 = G.make_params(W.bl600(G.SE), precision=G.FP64, level_min=level)
    G.stmc_estimate(eps, level, G.SE, p64, 7, n_pilot=4000, workspace=ws)   # warm-up
    ts = []
    for _ in range(repeats):
        torch.cuda.synchronize()
        t = time.perf_counter()
        s = G.stmc_estimate(eps, level, G.SE, p64, 7, n_pilot=4000, workspace=ws)
        ts.append(time.perf_counter() - t)
    sp = _spread(ts)
    out["stmc_fp64_se"] = {"seconds": sp["median"], "seconds_spread": sp, "level": level,
                           "M": 8 << level, "N": s["N"][0], "estimate_m": s["estimate"][0],
                           "rmse_stat_m": math.sqrt(s["est_variance"][0]),
                           "path_steps": s["total_path_steps"]}
    out["mlmc_fp32_se_graph_level"] = level
    out["speedup"] = sp["median"] / dt if dt > 0 else None
    return out


def serving(n=500, rate_hz=200.0):
    """The serving workload: n queries arriving as a Poisson stream at rate_hz
    (u* ~ U[0.1, 0.5] m/s, H ~ U[300, 1500] m, z0/H ~ U[0.01, 0.5],
    T ~ U[300, 3600] s, eps/H in {2^-6, 2^-8, 2^-10}, BAOAB, FP32 paths)
    served in real time; latency is submit-to-finish."""
    from paper_1612_07717_gb300 import serve as S
    S.run(n=40, rate_hz=rate_hz, seed=3)            # warm-up: module loads, pinned buffers
    summary, results, _ = S.run(n=n, rate_hz=rate_hz, seed=7)
    summary["statuses"] = {str(k): sum(r["status"] == k for r in results)
                           for k in sorted({r["status"] for r in results})}
    summary["workload"] = ("Poisson arrivals; u*~U[0.1,0.5] m/s, H~U[300,1500] m, z0/H~U[0.01,0.5],"
                           " T~U[300,3600] s, eps/H in {2^-6,2^-8,2^-10}; BAOAB, FP32 paths")
    return summary


def adaptive_cost(G, W, torch, eps=1e-4, x_adapt=0.05):
    """Section 7.3's comparison in the paper's scenario: MLMC to RMSE eps on
    E[X_T] with uniform and with adaptive timesteps (X_adapt = 0.05), SE and
    GL, FP32 paths, host-driven estimator; plus the adaptive kernel's
    throughput on one level against the uniform kernel's."""
    out = {"eps": eps, "x_adapt": x_adapt, "scenario": "paper (H = 1, T = 1, X0 = 0.05)"}
    for name, integ in (("se", G.SE), ("gl", G.GL)):
        row = {}
        for mode, za in (("uniform", 0.0), ("adaptive", x_adapt)):
            p = G.make_params(dict(W.PAPER, z_adapt=za, L_max=12), precision=G.FP32)
            ws = G.Workspace(p)
            G.estimate(eps * 4, integ, p, 2, workspace=ws)   # warm-up
            torch.cuda.synchronize()
            t = time.perf_counter()
            r = G.estimate(eps, integ, p, 3, workspace=ws)
            dt = time.perf_counter() - t
            level = 6
            n = 1 << 20
            G.level_sums(level, n, integ, p, 4, workspace=ws)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            s = G.level_sums(level, n, integ, p, 4, workspace=ws)
            dt1 = time.perf_counter() - t1
            row[mode] = {"seconds": dt, "L": r["L"], "estimate": r["estimate"][0],
                         "path_steps": r["total_path_steps"], "converged": r["converged"],
                         "level6_path_steps_per_s": s["path_steps"] / dt1,
                         "level6_steps_per_pair": s["path_steps"] / n}
        out[name] = row
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-time-to-eps", action="store_true")
    ap.add_argument("--no-adaptive", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--n0", type=float, default=N0)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import ctypes as C
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_07717_gb300 as G
    from paper_1612_07717_gb300 import autotune
    from paper_1612_07717_gb300 import workloads as W

    tuned = autotune.apply()            # the autotuner's table for this GPU, if recorded
    tuning = dict(autotune.get_tuning(INTEGRATOR, G.FP32),
                  source="autotuner table" if tuned else "library defaults")

    # each rank takes its own slice of every level's path range (weak scaling:
    # the per-GPU work is the full schedule; ranks use disjoint path indices)
    sched = [(l, int(round(n * args.n0 / N0))) for l, n in workload()]
    reqs = [(l, rank * n, n) for l, n in sched]
    params = G.make_params(W.bl600(INTEGRATOR), precision=G.FP32)
    steps_per_step = path_steps_of(sched)
    launch = G.MultilevelLaunch(reqs, INTEGRATOR, params, seed=1)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2

    for w in range(args.warmup):
        launch.run(stream)
    torch.cuda.synchronize()

    import tempfile
    clk_file = os.path.join(tempfile.gettempdir(),
                            "mlmc_bench_clocks_rank%d_%d.csv" % (rank, os.getpid()))
    sampler = sample_clocks(None, clk_file) if rank == 0 else None
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    times = []
    for k in range(args.steps):
        flush.zero_()                              # L2 flush outside the timed events
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        launch.run(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    if sampler:
        sampler.terminate()
        sampler.wait()
    ms = sum(times) / len(times)
    t_max = torch.tensor([ms], device="cuda")
    if world > 1:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    ms = float(t_max.item())
    res = launch.results()
    assert all(r["n"] == c for r, (_, _, c) in zip(res, launch.requests)), "lost paths"

    # end to end through the public C ABI with host requests and host results
    e2e_times = []
    reqs_host = list(launch.requests)
    for k in range(max(2, args.steps // 2)):
        t = time.perf_counter()
        G.multilevel_sums(reqs_host, INTEGRATOR, params, 1, workspace=launch.ws)
        e2e_times.append(time.perf_counter() - t)
    e2e_s = statistics.median(e2e_times)

    clocks = parse_clocks(clk_file) if rank == 0 else None
    peak_probe = fp32_peak_probe(torch)
    value = world * steps_per_step / (ms / 1e3)
    out = None
    if rank == 0:
        sm_mhz = clocks["sm_mhz"] if clocks else 2070.0
        info = G.device_info()
        derived_peak = info["sms"] * 128 * 2 * sm_mhz * 1e6
        peak = peak_probe or derived_peak
        achieved = FLOPS_PER_PATH_STEP * steps_per_step / (ms / 1e3)
        n_req = len(reqs_host)
        out = {
            "metric": "path-steps/s", "value": value, "unit": "path-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": dict(workload_config(sched), paths="fp32", sums="fp64 Kahan",
                           l2="flushed between timed steps (256 MB write)", tuning=tuning,
                           parallelism="replicas" if world > 1 else "single"),
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12,
                         "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": (TRAFFIC["bytes_per_launch"]
                                     if TRAFFIC["kernel_sha1"] == kernel_sha1() else None),
                         "peak_source": "measured FFMA probe" if peak_probe else
                         "derived SMs*128*2*clock at %.0f MHz" % sm_mhz,
                         "flops_per_path_step": FLOPS_PER_PATH_STEP,
                         "ncu": ({k: TRAFFIC[k] for k in ("fma_pipe_active_pct",
                                                          "fmaheavy_pipe_active_pct",
                                                          "issue_active_pct",
                                                          "thread_inst_per_path_step")}
                                 if TRAFFIC["kernel_sha1"] == kernel_sha1() else None),
                         # one instruction per SM sub-partition per cycle at the
                         # sampled clock: the path-steps/s the issue slots allow
                         "issue_ceiling_path_steps_per_s": (
                             info["sms"] * 4 * sm_mhz * 1e6 * 32 / TRAFFIC["thread_inst_per_path_step"]
                             if TRAFFIC["kernel_sha1"] == kernel_sha1() else None)},
            "e2e": {"value": world * steps_per_step / e2e_s, "unit": "path-steps/s",
                    "h2d_bytes_per_step": C.sizeof(G.LevelRequest) * n_req + C.sizeof(G.Params),
                    "d2h_bytes_per_step": C.sizeof(G.LevelResult) * n_req},
            "gpu_launches": 2 * args.steps,
            "clocks": clocks,
        }
        if not args.no_time_to_eps:
            out["time_to_eps"] = time_to_eps(G, W, torch)
        if not args.no_adaptive:
            out["adaptive_timesteps"] = adaptive_cost(G, W, torch)
        if not args.no_serving:
            out["serving"] = serving()
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline_sample()
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
