"""Autotuner of the persistent multi-level launch.

For each (integrator, precision) it times the batched workload (all levels
0..12 of the 600 m boundary layer, N_l = n0 * 10^(-l/2); n0 = 1e9 for FP32 by
default, the benchmark's own size, since the best item size depends on the
total work; SE, whose hierarchy starts at level 6, runs levels 6..12 scaled to
the same path-steps) for every combination of

* kernel variant: one path pair per thread, compiled for 1 (uncapped), 3 or
  4 resident 256-thread blocks per SM, or two pairs per thread on the packed
  FP32 instructions (12, 13: compiled for 2 or 3 blocks per SM);
* items per resident block: how finely the planner splits each level into
  work items, i.e. how many path pairs one thread integrates per item
  (paths per thread = item paths / 256);

keeps the first combination in sweep order (simpler variant, then fewer
items) whose rate is within 1 % of the fastest -- closer rates are within
run-to-run noise -- and records it as JSON keyed by the GPU name.  ``apply``
loads such a file into the library's tuning table (``mlmc_set_tuning``).
"""
import ctypes as C
import json
import os
import time

from . import BAOAB, FP32, FP64, GL, SE, MultilevelLaunch, lib, make_params
from . import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_FILE = os.path.join(HERE, "tuning_gb300.json")
VARIANTS = {FP32: (1, 3, 4, 12, 13), FP64: (1,)}
ITEMS_PER_BLOCK = (4, 8, 16, 32, 64)


def gpu_name():
    import torch
    return torch.cuda.get_device_name(0)


def set_tuning(integrator, precision, variant, items_per_block, blocks_per_sm=0):
    rc = lib().mlmc_set_tuning(integrator, precision, variant, items_per_block, blocks_per_sm)
    if rc != 0:
        raise ValueError("mlmc_set_tuning rejected %r" % ((integrator, precision, variant,
                                                            items_per_block, blocks_per_sm),))


def get_tuning(integrator, precision):
    out = (C.c_int32 * 3)()
    lib().mlmc_get_tuning(integrator, precision, out)
    return dict(variant=out[0], items_per_block=out[1], blocks_per_sm=out[2])


def _steps(sched, lm):
    """Path-steps of a schedule: 8 * 2^l fine steps per pair, plus the coupled
    coarse path's half as many above the base level."""
    return sum(n * ((8 << l) * 3 // 2 if l > lm else (8 << l)) for l, n in sched)


def tuning_schedule(integrator, n0):
    """[(level, N_l)] of the tuned launch: levels level_min..12 of the BL600
    hierarchy with N_l = n0 * 10^(-l/2).  A hierarchy that starts above level 0
    (SE's stable base level) has its counts scaled up to the path-steps of the
    levels-0..12 launch: cut to its finer levels alone, the launch would be so
    short that the finest level's pairs -- tens of thousands of steps each,
    sharing their warp scheduler with every other resident warp -- outlast the
    rest of the work, and the sweep would rank how the work items happened to
    land on the SMs rather than throughput."""
    lm = W.bl600(integrator)["level_min"]
    full = [(l, max(1, int(round(n * n0 / 1e9)))) for l, n in W.schedule_c4(levels=13, n0=1e9)]
    sched = [(l, n) for l, n in full if l >= lm]
    if lm > 0:
        f = _steps(full, 0) / _steps(sched, lm)
        sched = [(l, max(1, int(round(n * f)))) for l, n in sched]
    return sched


def _time_launch(integrator, precision, n0, reps=3):
    import torch
    d = W.bl600(integrator)
    lm = d["level_min"]
    sched = tuning_schedule(integrator, n0)
    p = make_params(d, precision=precision)
    launch = MultilevelLaunch([(l, 0, n) for l, n in sched], integrator, p, seed=1)
    steps = _steps(sched, lm)
    launch.run()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        launch.run()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return steps / (best / 1e3)


def select(results, tolerance=0.01):
    """(rate, variant, items_per_block) of the first entry, in sweep order,
    within `tolerance` of the best rate."""
    best = max(r for r, _, _ in results)
    return next(row for row in results if row[0] >= (1.0 - tolerance) * best)


def tune(integrators=(SE, GL, BAOAB), precisions=(FP32,), n0=1e9, verbose=False):
    """Sweep the launch knobs; returns {key: best config and rate} and applies the best."""
    out = {}
    for prec in precisions:
        for integ in integrators:
            scale = n0 if prec == FP32 else n0 / 100.0
            results = []
            for var in VARIANTS[prec]:
                for ipb in ITEMS_PER_BLOCK:
                    set_tuning(integ, prec, var, ipb, 0)
                    rate = _time_launch(integ, prec, scale)
                    results.append((rate, var, ipb))
                    if verbose:
                        print("integ %d prec %d variant %d items/block %d: %.3e path-steps/s"
                              % (integ, prec, var, ipb, rate), flush=True)
            rate, var, ipb = select(results)
            set_tuning(integ, prec, var, ipb, 0)
            out["%d/%d" % (integ, prec)] = dict(variant=var, items_per_block=ipb, blocks_per_sm=0,
                                                path_steps_per_s=rate,
                                                sweep=[dict(variant=v, items_per_block=i,
                                                            path_steps_per_s=r)
                                                       for r, v, i in results])
    return out


def save(table, path=DEFAULT_FILE):
    doc = dict(gpu=gpu_name(), when=time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()),
               workload="levels level_min..12, N_l = n0 10^(-l/2), BL600 scenario, "
               "n0 = 1e9 (FP32), 1e7 (FP64); SE (level_min 6) scaled to the "
               "path-steps of levels 0..12", table=table)
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)
    return path


def apply(path=DEFAULT_FILE, require_gpu_match=True):
    """Load a tuning file into the library; returns the table or None."""
    if not os.path.exists(path):
        return None
    doc = json.load(open(path))
    if require_gpu_match and doc.get("gpu") != gpu_name():
        return None
    for key, cfg in doc["table"].items():
        integ, prec = (int(x) for x in key.split("/"))
        set_tuning(integ, prec, cfg["variant"], cfg["items_per_block"], cfg.get("blocks_per_sm", 0))
    return doc["table"]


if __name__ == "__main__":
    import sys
    t = tune(precisions=(FP32, FP64), verbose=True)
    print(save(t, sys.argv[1] if len(sys.argv) > 1 else DEFAULT_FILE))
