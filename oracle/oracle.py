"""ctypes wrapper of the C oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: used by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``.  It imports nothing from the CUDA
package; parameters arrive as plain dicts.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

SE, GL, BAOAB = 0, 1, 2
U23, U32 = 0, 1
MAX_LEVELS = 32


class Params(C.Structure):
    _fields_ = [
        ("u_star", C.c_double), ("f_coriolis", C.c_double), ("H", C.c_double),
        ("kappa_sigma", C.c_double), ("kappa_tau", C.c_double), ("c_f", C.c_double),
        ("eps_reg_frac", C.c_double), ("z0", C.c_double), ("w0", C.c_double),
        ("T", C.c_double), ("qoi_threshold", C.c_double),
        ("w0_mode", C.c_int32), ("M0", C.c_int32), ("level_min", C.c_int32),
        ("L_max", C.c_int32), ("coupling", C.c_int32), ("drift_outside", C.c_int32),
        ("n_init", C.c_int32), ("uniform_map", C.c_int32), ("stream_id", C.c_uint32),
        ("qoi1_mode", C.c_int32), ("qoi_a", C.c_double), ("qoi_b", C.c_double),
        ("smooth_delta", C.c_double), ("smooth_r", C.c_int32), ("adapt_q", C.c_int32),
        ("z_adapt", C.c_double),
    ]


class PathOut(C.Structure):
    _fields_ = [("zf", C.c_double), ("wf", C.c_double), ("zc", C.c_double), ("wc", C.c_double),
                ("nonfinite", C.c_int32), ("refl_f", C.c_int32), ("refl_c", C.c_int32),
                ("pad_", C.c_int32), ("steps_f", C.c_int64), ("steps_c", C.c_int64),
                ("tie", C.c_double), ("gap", C.c_double)]


class LevelSums(C.Structure):
    _fields_ = [("n", C.c_uint64), ("path_steps", C.c_uint64), ("n_nonfinite", C.c_uint64),
                ("pad_", C.c_uint64), ("sum", (C.c_double * 6) * 2)]


class Result(C.Structure):
    _fields_ = [("estimate", C.c_double * 2), ("est_variance", C.c_double * 2),
                ("L", C.c_int32), ("converged", C.c_int32),
                ("N", C.c_uint64 * MAX_LEVELS), ("V", C.c_double * MAX_LEVELS),
                ("mean_y", C.c_double * MAX_LEVELS), ("total_path_steps", C.c_uint64),
                ("n_nonfinite", C.c_uint64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
        L.orc_philox4x32_10.restype = None
        L.orc_normals4.argtypes = [C.POINTER(Params), C.c_int, C.c_uint64, C.c_uint32,
                                   C.c_uint64, C.POINTER(C.c_double)]
        L.orc_normals4.restype = None
        L.orc_coefficients.argtypes = [C.POINTER(Params), C.c_double, C.POINTER(C.c_double)]
        L.orc_coefficients.restype = None
        L.orc_normalise.argtypes = [C.POINTER(Params)]
        L.orc_path.argtypes = [C.POINTER(Params), C.c_int, C.c_int, C.c_uint64, C.c_uint64,
                               C.POINTER(PathOut), C.c_void_p, C.c_void_p]
        L.orc_path_half.argtypes = [C.POINTER(Params), C.c_int, C.c_int, C.c_uint64, C.c_uint64,
                                    C.POINTER(PathOut), C.c_void_p, C.c_void_p]
        L.orc_level_sums.argtypes = [C.POINTER(Params), C.c_int, C.c_int, C.c_uint64,
                                     C.c_uint64, C.c_uint64, C.c_int, C.POINTER(LevelSums)]
        L.orc_smooth_poly.argtypes = [C.c_int, C.POINTER(C.c_double)]
        L.orc_g.argtypes = [C.c_int, C.POINTER(C.c_double), C.c_double]
        L.orc_g.restype = C.c_double
        L.orc_level_pdf_sums.argtypes = [C.POINTER(Params), C.c_int, C.c_int, C.c_uint64, C.c_uint64,
                                         C.c_uint64, C.c_int, C.c_int, C.POINTER(C.c_uint64),
                                         C.POINTER(C.c_double)]
        L.orc_estimate.argtypes = [C.POINTER(Params), C.c_int, C.c_double, C.c_uint64,
                                   C.c_int, C.POINTER(Result)]
        _lib = L
    return _lib


_DEFAULTS = dict(u_star=0.2, f_coriolis=1e-4, H=0.0, kappa_sigma=1.3, kappa_tau=0.5, c_f=0.0,
                 eps_reg_frac=1e-3, z0=0.0, w0=0.0, T=1.0, qoi_threshold=0.0, w0_mode=0, M0=8,
                 level_min=0, L_max=10, coupling=0, drift_outside=0, n_init=10000,
                 uniform_map=U32, stream_id=0, qoi1_mode=0, qoi_a=0.0, qoi_b=0.0,
                 smooth_delta=0.0, smooth_r=4, z_adapt=0.0, adapt_q=0)


def make_params(d=None, **kw):
    """Oracle parameter struct from a dict of the scenario fields."""
    vals = dict(_DEFAULTS)
    if d:
        vals.update({k: v for k, v in d.items() if k in _DEFAULTS})
    vals.update({k: v for k, v in kw.items() if k in _DEFAULTS})
    p = Params()
    for k, v in vals.items():
        setattr(p, k, v)
    if lib().orc_normalise(C.byref(p)) != 0:
        raise ValueError("invalid oracle parameters: %r" % (vals,))
    return p


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def normals4(p, level, i, block, seed):
    out = (C.c_double * 4)()
    lib().orc_normals4(C.byref(p), level, i, block, seed, out)
    return np.array(out[:])


def coefficients(p, z):
    """(sigma_w, sigma_w^2, d sigma_w^2/dz, lambda, sigma) at height z."""
    out = (C.c_double * 5)()
    lib().orc_coefficients(C.byref(p), float(z), out)
    return np.array(out[:])


def path(p, integ, level, i, seed, trace=False):
    """One path pair; with trace=True also the (z, w, S) rows of both paths."""
    r = PathOut()
    M = p.M0 << level
    tf = tc = None
    if trace:
        tf = np.zeros((M + 1, 3))
        tc = np.zeros((M // 2 + 1, 3))
    rc = lib().orc_path(C.byref(p), integ, level, i, seed, C.byref(r),
                        tf.ctypes.data if trace else None, tc.ctypes.data if trace else None)
    if rc != 0:
        raise ValueError("orc_path rejected its arguments")
    out = dict(zf=r.zf, wf=r.wf, zc=r.zc, wc=r.wc, nonfinite=r.nonfinite,
               refl_f=r.refl_f, refl_c=r.refl_c, steps_f=r.steps_f, steps_c=r.steps_c, tie=r.tie,
               gap=r.gap)
    if trace:
        out["trace_f"] = tf
        out["trace_c"] = tc
    return out


def path_half(p, integ, level, i, seed):
    """BAOAB pair with the (z, w, S) rows after the first half of every step
    (the fold that follows the first A half-step): half_f (M rows) and
    half_c (M/2 rows; zeros on the coarsest level)."""
    r = PathOut()
    M = p.M0 << level
    hf = np.zeros((M, 3))
    hc = np.zeros((M // 2, 3))
    rc = lib().orc_path_half(C.byref(p), integ, level, i, seed, C.byref(r), hf.ctypes.data,
                             hc.ctypes.data)
    if rc != 0:
        raise ValueError("orc_path_half rejected its arguments")
    return dict(zf=r.zf, wf=r.wf, zc=r.zc, wc=r.wc, nonfinite=r.nonfinite, half_f=hf,
                half_c=hc)


def paths(p, integ, level, N, offset, seed, extra=False):
    """Final states of N consecutive path pairs as an (N, 4) array plus flags;
    with extra=True also (steps_f, steps_c) per pair and the (tie, gap) margins."""
    zs = np.zeros((N, 4))
    bad = np.zeros(N, dtype=np.int32)
    steps = np.zeros((N, 2), dtype=np.int64)
    tie = np.zeros((N, 2))
    r = PathOut()
    for j in range(N):
        if lib().orc_path(C.byref(p), integ, level, offset + j, seed, C.byref(r), None, None):
            raise ValueError("orc_path rejected its arguments")
        zs[j] = (r.zf, r.wf, r.zc, r.wc)
        bad[j] = r.nonfinite
        steps[j] = (r.steps_f, r.steps_c)
        tie[j] = (r.tie, r.gap)
    if extra:
        return zs, bad, steps, tie
    return zs, bad


def level_sums(p, integ, level, N, offset=0, seed=1, threads=None):
    if threads is None:
        threads = os.cpu_count() or 1
    r = LevelSums()
    rc = lib().orc_level_sums(C.byref(p), integ, level, N, offset, seed, threads, C.byref(r))
    if rc != 0:
        raise ValueError("orc_level_sums rejected its arguments")
    return dict(n=r.n, path_steps=r.path_steps, n_nonfinite=r.n_nonfinite,
                sum=np.array([[r.sum[q][j] for j in range(6)] for q in range(2)]))


def estimate(p, integ, eps, seed=1, threads=None):
    if threads is None:
        threads = os.cpu_count() or 1
    r = Result()
    rc = lib().orc_estimate(C.byref(p), integ, eps, seed, threads, C.byref(r))
    if rc != 0:
        raise ValueError("orc_estimate rejected its arguments")
    L = r.L
    lm = p.level_min
    return dict(estimate=list(r.estimate), est_variance=list(r.est_variance), L=L,
                converged=r.converged, N=[r.N[l] for l in range(lm, L + 1)],
                V=[r.V[l] for l in range(lm, L + 1)],
                mean_y=[r.mean_y[l] for l in range(lm, L + 1)],
                total_path_steps=r.total_path_steps, n_nonfinite=r.n_nonfinite)


def smooth_poly(r):
    """Coefficients c_0..c_{r+1} of the smoothing polynomial p_r."""
    c = (C.c_double * (r + 2))()
    if lib().orc_smooth_poly(r, c) != 0:
        raise ValueError("orc_smooth_poly failed for r=%d" % r)
    return np.array(c[:])


def g(r, coef, x):
    c = (C.c_double * (r + 2))(*coef)
    return lib().orc_g(r, c, float(x))


def level_pdf_sums(p, integ, level, N, k, offset=0, seed=1, threads=None):
    if threads is None:
        threads = os.cpu_count() or 1
    out = (C.c_double * (6 * k))()
    n = C.c_uint64()
    rc = lib().orc_level_pdf_sums(C.byref(p), integ, level, N, offset, seed, k, threads,
                                  C.byref(n), out)
    if rc != 0:
        raise ValueError("orc_level_pdf_sums rejected its arguments")
    return dict(n=n.value, sum=np.array(out[:]).reshape(k, 6))
