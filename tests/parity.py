"""Helpers shared by the GPU parity tests: build matching parameter sets for
the CUDA library and the oracle from one workload dict, run both, and compare
per path with the reflection near-tie rule.

Tolerances (per path, final position):
  FP32 paths: |z_gpu - z_oracle| <= 1e-4 H.  A path may be exempt only when
    the two disagree on a reflection decision: at the first row where the
    parities differ the oracle's path is within 1e-5 H of a wall.  For BAOAB
    the rows include the state after the first half of every step (GPU and
    oracle half-step traces), so every fold has its row: a fold taken half a
    step apart on the two sides, which the full-step rows alone hide, is
    located exactly.  At most 1e-3 of the paths (and at least 2) may be
    exempt.
  FP64 paths: |dz| <= 1e-9 H, same exemption rule.
"""
import numpy as np

from oracle import oracle as O

import paper_1612_07717_gb300 as G


def gpu_params(d, precision=G.FP32, **kw):
    return G.make_params(d, precision=precision, **kw)


def oracle_params(d, precision=G.FP32, **kw):
    umap = O.U23 if precision == G.FP32 else O.U32
    return O.make_params(d, uniform_map=umap, **kw)


def tolerance(precision, H):
    return (1e-4 if precision == G.FP32 else 1e-9) * H


def _interleave(full, half):
    """Full-step rows and BAOAB's half-step rows in time order: full 0, half 0,
    full 1, half 1, ..., full M (row r at time r / 2 steps)."""
    out = np.empty((full.shape[0] + half.shape[0], full.shape[1]))
    out[0::2] = full
    out[1::2] = half
    return out


def near_tie(d, integ, level, i, seed, precision, tol):
    """True when path pair i differs only through a reflection near-tie: the
    two first disagree on a parity at a fold that left the oracle's path
    within 1e-5 H of a wall, and their positions had not separated before.
    For BAOAB the rows after each first half-step are included on both sides,
    so every fold of the path has a row."""
    pg = gpu_params(d, precision)
    po = oracle_params(d, precision)
    H = po.H
    tf, tc = G.path_trace(level, 1, integ, pg, seed, path_offset=i)
    tf = tf[0].double().cpu().numpy()
    tc = tc[0].double().cpu().numpy()
    r = O.path(po, integ, level, i, seed, trace=True)
    of, oc = r["trace_f"], r["trace_c"]
    coupled = level > po.level_min
    unit_f, unit_c = 1.0, 2.0            # fine steps per row
    if integ == O.BAOAB:
        hf, hc = G.path_trace_half(level, 1, integ, pg, seed, path_offset=i)
        rh = O.path_half(po, integ, level, i, seed)
        tf = _interleave(tf, hf[0].double().cpu().numpy())
        of = _interleave(of, rh["half_f"])
        tc = _interleave(tc, hc[0].double().cpu().numpy())
        oc = _interleave(oc, rh["half_c"])
        unit_f, unit_c = 0.5, 1.0
    # (gpu rows, oracle rows, fine steps per row)
    pairs = [(tf, of, unit_f)]
    if coupled:
        pairs.append((tc, oc, unit_c))
    flips, devs = [], []
    for g, o, unit in pairs:
        ds = g[:, 2] != o[:, 2]
        if ds.any():
            k = int(np.argmax(ds))          # the fold of row k is where the parities part
            flips.append((k * unit, o[k, 0]))
        dz = np.abs(g[:, 0] - o[:, 0]) > tol
        if dz.any():
            devs.append(int(np.argmax(dz)) * unit)
    if not devs:
        return False
    if not flips:
        return False            # positions separated with no reflection disagreement
    t_flip, z = min(flips)
    if min(devs) < t_flip:
        return False            # separated before the first parity flip
    win = 1e-5 * H
    return bool(z < win or H - z < win)


def compare_paths(d, integ, level, N, offset=0, seed=1, precision=G.FP32, max_exempt=None,
                  variant=None):
    """Run N pairs on both sides (the GPU side through tuning variant
    `variant`'s path code when given); return (max |dz| over non-exempt,
    n_exempt, gpu states, gpu flags, oracle states)."""
    pg = gpu_params(d, precision)
    po = oracle_params(d, precision)
    H = po.H
    tol = tolerance(precision, H)
    states, flags = G.level_paths(level, N, integ, pg, seed, path_offset=offset, variant=variant)
    gs = states.double().cpu().numpy()
    gf = flags.cpu().numpy()
    os_, of = O.paths(po, integ, level, N, offset, seed)
    assert np.array_equal(gf != 0, of != 0), "divergence flags differ"
    ok = gf == 0
    coupled = level > po.level_min
    dz = np.abs(gs[:, 0] - os_[:, 0])
    if coupled:
        dz = np.maximum(dz, np.abs(gs[:, 2] - os_[:, 2]))
    dz[~ok] = 0.0
    bad = np.nonzero(dz > tol)[0]
    exempt = []
    for j in bad:
        if near_tie(d, integ, level, offset + int(j), seed, precision, tol):
            exempt.append(int(j))
        else:
            raise AssertionError("path %d: |dz| = %.3e > %.3e (gpu %s, oracle %s)"
                                 % (offset + j, dz[j], tol, gs[j], os_[j]))
    if max_exempt is None:
        max_exempt = max(2, int(1e-3 * N))
    assert len(exempt) <= max_exempt, "too many near-tie exemptions: %d" % len(exempt)
    dz[exempt] = 0.0
    return float(dz.max(initial=0.0)), len(exempt), gs, gf, os_


def sums_from_states(gs, gf, thr, coupled, precision):
    """Level sums recomputed in float64 from per-path states (the reduction
    kernel must reproduce these; counts exactly)."""
    ok = gf == 0
    zf = gs[ok, 0]
    zc = gs[ok, 2] if coupled else np.zeros_like(zf)
    dt = np.float32 if precision == G.FP32 else np.float64
    If = (zf.astype(dt) < dt(thr)).astype(np.float64)
    Ic = ((zc.astype(dt) < dt(thr)) & coupled).astype(np.float64)
    out = []
    for Pf, Pc in ((zf, zc), (If, Ic)):
        Y = Pf - Pc
        out.append([Y.sum(), (Y * Y).sum(), Pf.sum(), (Pf * Pf).sum(), Pc.sum(), (Pc * Pc).sum()])
    return dict(n=int(ok.sum()), n_nonfinite=int((~ok).sum()), sum=np.array(out))
