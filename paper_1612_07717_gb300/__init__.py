"""GB300 (sm_103a) multilevel Monte Carlo for 1-D boundary-layer dispersion.

Thin ctypes binding over the C ABI of ``libmlmc.so`` (declared in
``include/mlmc.h``): argument marshalling only; every step of the path runs
in the library's CUDA kernels.  PyTorch supplies device memory (the
workspace and output tensors) and streams.  Importing the package does not
load the library; the first call does, and it raises if the library has not
been built -- there is no CPU fallback.

Method: Katsiolides, Mueller, Scheichl, Shardlow, Giles, Thomson, "Multilevel
Monte Carlo and improved timestepping methods in atmospheric dispersion
modelling", arXiv 1612.07717.
"""
import ctypes as C
import os

from . import workloads  # noqa: F401  (inputs only; no library load)

SE, GL, BAOAB = 0, 1, 2
FP32, FP64 = 0, 1
MAX_LEVELS = 32

OK, EINVAL, EWORKSPACE, ECUDA, ENONFINITE, ETIMEOUT, EUNSTABLE, ENOTCONV, ENODEV, ECOMM = (
    0, -1, -2, -3, -4, -5, -6, -7, -8, -9)

# reduce hook of mlmc_estimate_sharded: int (*)(double* buf, int n, void* ctx)
ALLREDUCE_FN = C.CFUNCTYPE(C.c_int, C.POINTER(C.c_double), C.c_int, C.c_void_p)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmlmc.so")


class Params(C.Structure):
    """mirror of ``mlmc_params`` (include/mlmc.h)"""
    _fields_ = [
        ("u_star", C.c_double), ("f_coriolis", C.c_double), ("H", C.c_double),
        ("kappa_sigma", C.c_double), ("kappa_tau", C.c_double), ("c_f", C.c_double),
        ("eps_reg_frac", C.c_double), ("z0", C.c_double), ("w0", C.c_double),
        ("T", C.c_double), ("qoi_threshold", C.c_double),
        ("w0_mode", C.c_int32), ("M0", C.c_int32), ("level_min", C.c_int32),
        ("L_max", C.c_int32), ("coupling", C.c_int32), ("drift_outside", C.c_int32),
        ("n_init", C.c_int32), ("precision", C.c_int32), ("stream_id", C.c_uint32),
        ("allow_unstable", C.c_int32), ("qoi1_mode", C.c_int32), ("smooth_r", C.c_int32),
        ("qoi_a", C.c_double), ("qoi_b", C.c_double), ("smooth_delta", C.c_double),
        ("z_adapt", C.c_double),
    ]


class LevelResult(C.Structure):
    _fields_ = [("n", C.c_uint64), ("path_steps", C.c_uint64), ("n_nonfinite", C.c_uint64),
                ("reserved", C.c_uint64), ("sum", (C.c_double * 6) * 2)]


class Result(C.Structure):
    _fields_ = [("estimate", C.c_double * 2), ("est_variance", C.c_double * 2),
                ("L", C.c_int32), ("converged", C.c_int32),
                ("N", C.c_uint64 * MAX_LEVELS), ("V", C.c_double * MAX_LEVELS),
                ("mean_y", C.c_double * MAX_LEVELS), ("total_path_steps", C.c_uint64),
                ("n_nonfinite", C.c_uint64), ("seconds", C.c_double)]


class EstimateState(C.Structure):
    """``mlmc_estimate_state``: the host-driven estimator's whole state."""
    _fields_ = [("eps", C.c_double), ("seed", C.c_uint64), ("integrator", C.c_int32),
                ("L", C.c_int32), ("phase", C.c_int32), ("converged", C.c_int32),
                ("n_done", C.c_uint64 * MAX_LEVELS), ("n", C.c_uint64 * MAX_LEVELS),
                ("n_nonfinite", C.c_uint64 * MAX_LEVELS),
                ("path_steps", C.c_uint64 * MAX_LEVELS),
                ("sum", ((C.c_double * 6) * 2) * MAX_LEVELS), ("seconds", C.c_double),
                ("passes", C.c_int32), ("reserved", C.c_int32)]


class LevelRequest(C.Structure):
    _fields_ = [("level", C.c_int32), ("reserved", C.c_int32), ("first", C.c_uint64),
                ("count", C.c_uint64)]


assert C.sizeof(Params) == 168 and C.sizeof(LevelResult) == 128


class MLMCError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s: %s (%d)" % (where, strerror(code), code))


_lib = None


def lib():
    """The loaded library; raises if it was not built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libmlmc.so not built: run paper_1612_07717_gb300.build.build() "
                               "(expected at %s)" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        vp, u64, i32 = C.c_void_p, C.c_uint64, C.c_int
        L.mlmc_strerror.restype = C.c_char_p
        L.mlmc_strerror.argtypes = [i32]
        L.mlmc_params_default.argtypes = [C.POINTER(Params)]
        L.mlmc_device_info.argtypes = [C.POINTER(C.c_int32)]
        L.mlmc_workspace_bytes.restype = C.c_size_t
        L.mlmc_workspace_bytes.argtypes = [C.POINTER(Params), i32]
        L.mlmc_level_sums.argtypes = [i32, u64, i32, C.POINTER(Params), u64, u64, vp, C.c_size_t,
                                      vp, C.POINTER(LevelResult)]
        L.mlmc_multilevel_sums_async.argtypes = [C.POINTER(LevelRequest), i32, i32,
                                                 C.POINTER(Params), u64, vp, C.c_size_t, vp, vp]
        L.mlmc_multilevel_sums.argtypes = [C.POINTER(LevelRequest), i32, i32, C.POINTER(Params),
                                           u64, vp, C.c_size_t, vp, C.POINTER(LevelResult)]
        L.mlmc_estimate.argtypes = [C.c_double, i32, C.POINTER(Params), u64, vp, C.c_size_t, vp,
                                    C.POINTER(Result)]
        L.mlmc_estimate_begin.argtypes = [C.c_double, i32, C.POINTER(Params), u64,
                                          C.POINTER(EstimateState)]
        L.mlmc_estimate_pass.argtypes = [C.POINTER(EstimateState), C.POINTER(Params), vp,
                                         C.c_size_t, vp]
        L.mlmc_estimate_result.argtypes = [C.POINTER(EstimateState), C.POINTER(Params),
                                           C.POINTER(Result)]
        L.mlmc_estimate_sharded.argtypes = [C.c_double, i32, C.POINTER(Params), u64, i32, i32,
                                            ALLREDUCE_FN, vp, vp, C.c_size_t, vp,
                                            C.POINTER(Result)]
        L.mlmc_graph_create.argtypes = [C.c_double, i32, C.POINTER(Params), u64, vp, C.c_size_t,
                                        C.POINTER(vp)]
        L.mlmc_graph_create_ex.argtypes = [C.c_double, i32, C.POINTER(Params), u64, i32, vp,
                                           C.c_size_t, C.POINTER(vp)]
        L.mlmc_graph_launch.argtypes = [vp, vp]
        L.mlmc_graph_result.argtypes = [vp, vp, C.POINTER(Result)]
        L.mlmc_graph_destroy.argtypes = [vp]
        L.mlmc_estimate_graph.argtypes = [C.c_double, i32, C.POINTER(Params), u64, vp, C.c_size_t,
                                          vp, C.POINTER(Result)]
        L.mlmc_level_pdf_sums.argtypes = [i32, u64, i32, C.POINTER(Params), u64, u64, i32, vp,
                                          C.c_size_t, vp, C.POINTER(C.c_double),
                                          C.POINTER(u64), C.POINTER(u64)]
        L.mlmc_estimate_pdf.argtypes = [C.c_double, i32, C.POINTER(Params), u64, i32, vp,
                                        C.c_size_t, vp, C.POINTER(C.c_double), C.POINTER(Result)]
        L.mlmc_stable_level_min.argtypes = [C.POINTER(Params), i32, C.POINTER(C.c_int32)]
        L.mlmc_multilevel_plan.argtypes = [C.POINTER(LevelRequest), i32, i32, C.POINTER(Params),
                                           i32, C.POINTER(C.c_uint32)]
        L.mlmc_set_tuning.argtypes = [i32, i32, i32, i32, i32]
        L.mlmc_get_tuning.argtypes = [i32, i32, C.POINTER(C.c_int32)]
        L.mlmc_server_workspace_bytes.restype = C.c_size_t
        L.mlmc_server_workspace_bytes.argtypes = [i32]
        L.mlmc_server_query_bytes.restype = C.c_size_t
        L.mlmc_server_query_bytes.argtypes = [C.POINTER(Params)]
        L.mlmc_server_pool.argtypes = [vp, C.POINTER(C.c_uint64)]
        L.mlmc_server_create.argtypes = [i32, i32, i32, u64, vp, C.c_size_t, vp, C.POINTER(vp)]
        L.mlmc_server_submit.argtypes = [vp, C.POINTER(Params), C.c_double, C.POINTER(u64)]
        L.mlmc_server_tick.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.mlmc_server_poll.argtypes = [vp, u64, C.POINTER(Result), C.POINTER(C.c_double)]
        L.mlmc_server_release.argtypes = [vp, u64]
        L.mlmc_server_stats.argtypes = [vp, C.POINTER(C.c_double)]
        L.mlmc_server_destroy.argtypes = [vp]
        L.mlmc_stmc_estimate.argtypes = [C.c_double, i32, i32, i32, C.POINTER(Params), u64, vp,
                                         C.c_size_t, vp, C.POINTER(Result)]
        L.mlmc_level_paths_async.argtypes = [i32, u64, i32, C.POINTER(Params), u64, u64, vp, vp, vp]
        L.mlmc_level_paths_variant_async.argtypes = [i32, i32, u64, i32, C.POINTER(Params), u64,
                                                     u64, vp, vp, vp]
        L.mlmc_level_paths_steps_async.argtypes = [i32, u64, i32, C.POINTER(Params), u64, u64, vp,
                                                   vp, vp, vp]
        L.mlmc_path_trace_async.argtypes = [i32, u64, i32, C.POINTER(Params), u64, u64, vp, vp, vp]
        L.mlmc_path_trace_half_async.argtypes = [i32, u64, i32, C.POINTER(Params), u64, u64, vp,
                                                 vp, vp]
        _lib = L
    return _lib


def strerror(code):
    try:
        return lib().mlmc_strerror(code).decode()
    except Exception:
        return "status %d" % code


def _check(rc, where, allow=()):
    if rc != OK and rc not in allow:
        raise MLMCError(rc, where)
    return rc


_PARAM_FIELDS = [f for f, _ in Params._fields_]


def make_params(d=None, **kw):
    """``Params`` from the library defaults, updated by a dict and keywords."""
    p = Params()
    lib().mlmc_params_default(C.byref(p))
    for src in (d or {}), kw:
        for k, v in src.items():
            if k in _PARAM_FIELDS:
                setattr(p, k, v)
    return p


def stable_level_min(params, integrator):
    """Smallest stable level of the hierarchy (symplectic Euler: h lambda_max < 2)."""
    out = C.c_int32()
    _check(lib().mlmc_stable_level_min(C.byref(params), integrator, C.byref(out)),
           "mlmc_stable_level_min")
    return out.value


def device_info():
    out = (C.c_int32 * 3)()
    _check(lib().mlmc_device_info(out), "mlmc_device_info")
    return dict(sms=out[0], cc=out[1], version=out[2])


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class Workspace:
    """Device scratch owned by the caller (a torch uint8 tensor, 256-B aligned)."""

    def __init__(self, params=None, max_requests=1, device=None):
        import torch
        p = params if params is not None else make_params()
        self.nbytes = int(lib().mlmc_workspace_bytes(C.byref(p), max_requests))
        dev = torch.device(device) if device is not None else torch.device("cuda")
        self._buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=dev)
        base = self._buf.data_ptr()
        self.ptr = (base + 255) // 256 * 256

    def args(self):
        return C.c_void_p(self.ptr), C.c_size_t(self.nbytes)


def _level_result(r):
    return dict(n=r.n, path_steps=r.path_steps, n_nonfinite=r.n_nonfinite,
                sum=[[r.sum[q][j] for j in range(6)] for q in range(2)])


def level_sums(level, N, integrator, params, seed, path_offset=0, workspace=None, stream=None):
    """Sums of N coupled pairs of one level (``mlmc_level_sums``)."""
    ws = workspace or Workspace(params)
    r = LevelResult()
    rc = lib().mlmc_level_sums(level, N, integrator, C.byref(params), seed, path_offset,
                               *ws.args(), _stream_handle(stream), C.byref(r))
    _check(rc, "mlmc_level_sums", allow=(ENONFINITE,))
    return _level_result(r)


def multilevel_sums(requests, integrator, params, seed, workspace=None, stream=None):
    """Sums of many levels in one persistent launch; requests = [(level, first, count)]."""
    n = len(requests)
    ws = workspace or Workspace(params, n)
    arr = (LevelRequest * n)()
    for k, (lvl, first, count) in enumerate(requests):
        arr[k].level, arr[k].first, arr[k].count = lvl, first, count
    out = (LevelResult * n)()
    rc = lib().mlmc_multilevel_sums(arr, n, integrator, C.byref(params), seed, *ws.args(),
                                    _stream_handle(stream), out)
    _check(rc, "mlmc_multilevel_sums", allow=(ENONFINITE,))
    return [_level_result(out[k]) for k in range(n)]


def multilevel_plan(requests, integrator, params, grid):
    """Work-item plan of a batched launch on `grid` blocks (host only): one dict
    per request in launch order (finest level first) with the request's index,
    paths per item, items, first item and whether the packed kernel runs it one
    pair per thread (``single``)."""
    n = len(requests)
    arr = (LevelRequest * n)()
    for k, (lvl, first, count) in enumerate(requests):
        arr[k].level, arr[k].first, arr[k].count = lvl, first, count
    out = (C.c_uint32 * (5 * n))()
    _check(lib().mlmc_multilevel_plan(arr, n, integrator, C.byref(params), grid, out),
           "mlmc_multilevel_plan")
    keys = ("request", "item_paths", "n_items", "item_base", "single")
    return [dict(zip(keys, out[5 * k:5 * k + 5])) for k in range(n)]


class MultilevelLaunch:
    """Preplanned asynchronous batched launch with device-resident results.

    ``run()`` enqueues the persistent kernel and the per-request reduction on
    the stream and returns without synchronising; ``results()`` copies the
    device results back.  Requests are sorted finest level first.
    """

    def __init__(self, requests, integrator, params, seed, workspace=None):
        import torch
        reqs = sorted(requests, key=lambda r: -r[0])
        self.requests = reqs
        self.n = len(reqs)
        self.integrator = integrator
        self.params = params
        self.seed = seed
        self.ws = workspace or Workspace(params, self.n)
        self.arr = (LevelRequest * self.n)()
        for k, (lvl, first, count) in enumerate(reqs):
            self.arr[k].level, self.arr[k].first, self.arr[k].count = lvl, first, count
        self.d_out = torch.zeros(self.n * C.sizeof(LevelResult), dtype=torch.uint8,
                                 device=torch.device("cuda"))

    def run(self, stream=None):
        rc = lib().mlmc_multilevel_sums_async(self.arr, self.n, self.integrator,
                                              C.byref(self.params), self.seed, *self.ws.args(),
                                              _stream_handle(stream),
                                              C.c_void_p(self.d_out.data_ptr()))
        _check(rc, "mlmc_multilevel_sums_async")

    def results(self):
        raw = self.d_out.cpu().numpy().tobytes()
        out = (LevelResult * self.n).from_buffer_copy(raw)
        return [_level_result(out[k]) for k in range(self.n)]


def _result(r, lmin):
    L = r.L
    return dict(estimate=list(r.estimate), est_variance=list(r.est_variance), L=L,
                converged=r.converged, N=[r.N[l] for l in range(lmin, L + 1)],
                V=[r.V[l] for l in range(lmin, L + 1)],
                mean_y=[r.mean_y[l] for l in range(lmin, L + 1)],
                total_path_steps=r.total_path_steps, n_nonfinite=r.n_nonfinite,
                seconds=r.seconds)


def estimate(eps, integrator, params, seed, workspace=None, stream=None):
    """Adaptive MLMC estimate to RMSE eps (``mlmc_estimate``)."""
    ws = workspace or Workspace(params)
    r = Result()
    rc = lib().mlmc_estimate(eps, integrator, C.byref(params), seed, *ws.args(),
                             _stream_handle(stream), C.byref(r))
    _check(rc, "mlmc_estimate", allow=(ENONFINITE, ENOTCONV))
    out = _result(r, params.level_min)
    out["status"] = rc
    return out


class Estimation:
    """The host-driven estimate one pass at a time (``mlmc_estimate_begin``,
    ``mlmc_estimate_pass``, ``mlmc_estimate_result``), with a JSON checkpoint
    of its state: ``state_dict`` / ``from_state_dict``, or ``run(checkpoint=
    path)`` which writes the state after every pass and resumes from the
    file when it exists.  A resumed run gives the uninterrupted result bit
    for bit (floats are written with their exact repr)."""

    def __init__(self, eps, integrator, params, seed, workspace=None, stream=None):
        self.params = params
        self.workspace = workspace or Workspace(params)
        self.stream = stream
        self.state = EstimateState()
        _check(lib().mlmc_estimate_begin(eps, integrator, C.byref(params), seed,
                                         C.byref(self.state)), "mlmc_estimate_begin")

    @property
    def done(self):
        return self.state.phase == 2

    def step(self):
        """Run the next pass; True once the estimate is complete."""
        rc = lib().mlmc_estimate_pass(C.byref(self.state), C.byref(self.params),
                                      *self.workspace.args(), _stream_handle(self.stream))
        if rc == 1:
            return True
        _check(rc, "mlmc_estimate_pass")
        return False

    def result(self):
        r = Result()
        rc = lib().mlmc_estimate_result(C.byref(self.state), C.byref(self.params), C.byref(r))
        _check(rc, "mlmc_estimate_result", allow=(ENONFINITE, ENOTCONV))
        out = _result(r, self.params.level_min)
        out["status"] = rc
        return out

    def state_dict(self):
        st = self.state
        d = {}
        for name, _ in EstimateState._fields_:
            v = getattr(st, name)
            if name == "sum":
                d[name] = [[list(v[l][q]) for q in range(2)] for l in range(MAX_LEVELS)]
            elif isinstance(v, (int, float)):
                d[name] = v
            else:
                d[name] = list(v)
        return d

    def load_state_dict(self, d):
        st = EstimateState()
        for name, _ in EstimateState._fields_:
            v = d[name]
            if name == "sum":
                for l in range(MAX_LEVELS):
                    for q in range(2):
                        for k in range(6):
                            st.sum[l][q][k] = float(v[l][q][k])
            elif isinstance(v, list):
                arr = getattr(st, name)
                for k, x in enumerate(v):
                    arr[k] = x
            else:
                setattr(st, name, v)
        self.state = st

    def run(self, checkpoint=None):
        """Run to completion; with a checkpoint path, resume from it if it
        exists and rewrite it after every pass."""
        import json
        if checkpoint and os.path.exists(checkpoint):
            with open(checkpoint) as f:
                self.load_state_dict(json.load(f))
        while not self.done:
            self.step()
            if checkpoint:
                tmp = checkpoint + ".tmp"
                with open(tmp, "w") as f:
                    json.dump(self.state_dict(), f)
                os.replace(tmp, checkpoint)
        return self.result()


def rates(result, level_min=0):
    """Giles' MLMC rates from an estimate's per-level statistics: alpha with
    |E[Y_l]| ~ 2^(-alpha l) and beta with V_l ~ 2^(-beta l), least-squares
    slopes over the coupled levels (level_min + 1 .. L) whose values are
    positive; None where fewer than two levels qualify."""
    import math

    def slope(values):
        pts = [(level_min + k, math.log2(abs(v))) for k, v in enumerate(values)
               if k > 0 and v != 0.0]
        if len(pts) < 2:
            return None
        mx = sum(x for x, _ in pts) / len(pts)
        my = sum(y for _, y in pts) / len(pts)
        sxx = sum((x - mx) ** 2 for x, _ in pts)
        return -sum((x - mx) * (y - my) for x, y in pts) / sxx
    return dict(alpha=slope(result["mean_y"]), beta=slope(result["V"]))


def torch_allreduce(group=None):
    """A reduce hook for estimate_sharded over a torch.distributed group:
    the buffer goes through a float64 tensor on the group's device (CPU for
    gloo, the current CUDA device for nccl) and an all-reduce SUM."""
    import torch
    import torch.distributed as dist

    def reduce(values):
        dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
        t = torch.tensor(values, dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        return t.cpu().tolist()
    return reduce


def estimate_sharded(eps, integrator, params, seed, rank, world, reduce, workspace=None,
                     stream=None):
    """mlmc_estimate_sharded: this rank's share of every level, the sums
    combined by reduce(list of floats) -> list of their sums over ranks."""
    ws = workspace or Workspace(params)
    failed = []

    def hook(buf, n, ctx):
        try:
            vals = reduce([buf[k] for k in range(n)])
            for k in range(n):
                buf[k] = float(vals[k])
            return 0
        except Exception as e:          # reported to the library as a failed reduction
            failed.append(e)
            return 1
    cb = ALLREDUCE_FN(hook)
    r = Result()
    rc = lib().mlmc_estimate_sharded(eps, integrator, C.byref(params), seed, rank, world, cb,
                                     None, *ws.args(), _stream_handle(stream), C.byref(r))
    if failed:
        raise MLMCError(rc, "mlmc_estimate_sharded (reduce hook: %r)" % failed[0])
    _check(rc, "mlmc_estimate_sharded", allow=(ENONFINITE, ENOTCONV))
    out = _result(r, params.level_min)
    out["status"] = rc
    return out


def estimate_graph(eps, integrator, params, seed, workspace=None, stream=None):
    """Adaptive MLMC estimate with the loop captured in one CUDA graph."""
    ws = workspace or Workspace(params)
    r = Result()
    rc = lib().mlmc_estimate_graph(eps, integrator, C.byref(params), seed, *ws.args(),
                                   _stream_handle(stream), C.byref(r))
    _check(rc, "mlmc_estimate_graph", allow=(ENONFINITE, ENOTCONV))
    out = _result(r, params.level_min)
    out["status"] = rc
    return out


class GraphEstimator:
    """An instantiated graph of the adaptive loop, launched many times;
    max_passes > 0 lowers the device loop's pass limit (its watchdog)."""

    def __init__(self, eps, integrator, params, seed, workspace=None, max_passes=0):
        self.params = params
        self.ws = workspace or Workspace(params)
        self.handle = C.c_void_p()
        rc = lib().mlmc_graph_create_ex(eps, integrator, C.byref(params), seed, max_passes,
                                        *self.ws.args(), C.byref(self.handle))
        _check(rc, "mlmc_graph_create_ex")

    def launch(self, stream=None):
        _check(lib().mlmc_graph_launch(self.handle, _stream_handle(stream)), "mlmc_graph_launch")

    def result(self, stream=None):
        r = Result()
        rc = lib().mlmc_graph_result(self.handle, _stream_handle(stream), C.byref(r))
        _check(rc, "mlmc_graph_result", allow=(ENONFINITE, ENOTCONV))
        out = _result(r, self.params.level_min)
        out["status"] = rc
        return out

    def close(self):
        if self.handle:
            lib().mlmc_graph_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def level_pdf_sums(level, N, integrator, params, seed, k, path_offset=0, workspace=None,
                   stream=None):
    """Per-bin sums (sum Y_i, sum Y_i^2) of the binned density on one level."""
    ws = workspace or Workspace(params)
    out = (C.c_double * (2 * k))()
    nok, nbad = C.c_uint64(), C.c_uint64()
    rc = lib().mlmc_level_pdf_sums(level, N, integrator, C.byref(params), seed, path_offset, k,
                                   *ws.args(), _stream_handle(stream), out, C.byref(nok),
                                   C.byref(nbad))
    _check(rc, "mlmc_level_pdf_sums", allow=(ENONFINITE,))
    return dict(n=nok.value, n_nonfinite=nbad.value,
                sum=[[out[2 * i], out[2 * i + 1]] for i in range(k)])


def estimate_pdf(eps, integrator, params, seed, k, workspace=None, stream=None):
    """Adaptive MLMC estimate of the k-bin density (``mlmc_estimate_pdf``)."""
    ws = workspace or Workspace(params)
    pdf = (C.c_double * k)()
    r = Result()
    rc = lib().mlmc_estimate_pdf(eps, integrator, C.byref(params), seed, k, *ws.args(),
                                 _stream_handle(stream), pdf, C.byref(r))
    _check(rc, "mlmc_estimate_pdf", allow=(ENONFINITE, ENOTCONV))
    out = _result(r, params.level_min)
    out["pdf"] = list(pdf[:k])
    out["status"] = rc
    return out


def stmc_estimate(eps, level, integrator, params, seed, n_pilot=10000, workspace=None,
                  stream=None):
    """Plain Monte Carlo at level's timestep to RMSE eps (``mlmc_stmc_estimate``)."""
    ws = workspace or Workspace(params)
    r = Result()
    rc = lib().mlmc_stmc_estimate(eps, level, n_pilot, integrator, C.byref(params), seed,
                                  *ws.args(), _stream_handle(stream), C.byref(r))
    _check(rc, "mlmc_stmc_estimate", allow=(ENONFINITE,))
    out = _result(r, level)
    out["status"] = rc
    return out


def level_paths(level, N, integrator, params, seed, path_offset=0, stream=None, steps=False,
                variant=None):
    """Final (z_f, w_f, z_c, w_c) of N pairs as an (N, 4) CUDA tensor, plus flags;
    with steps=True (adaptive timesteps only) also the (N, 2) int64 step counts;
    with variant (0 = the tuning table's, or 1, 3, 4, 12, 13) through that
    tuning variant's path code (``mlmc_level_paths_variant_async``)."""
    import torch
    dt = torch.float64 if params.precision == FP64 else torch.float32
    states = torch.empty((N, 4), dtype=dt, device="cuda")
    flags = torch.empty(N, dtype=torch.int32, device="cuda")
    if variant is not None:
        rc = lib().mlmc_level_paths_variant_async(
            variant, level, N, integrator, C.byref(params), seed, path_offset,
            C.c_void_p(states.data_ptr()), C.c_void_p(flags.data_ptr()), _stream_handle(stream))
        _check(rc, "mlmc_level_paths_variant_async")
        return states, flags
    if steps:
        st = torch.empty((N, 2), dtype=torch.int64, device="cuda")
        rc = lib().mlmc_level_paths_steps_async(
            level, N, integrator, C.byref(params), seed, path_offset,
            C.c_void_p(states.data_ptr()), C.c_void_p(flags.data_ptr()),
            C.c_void_p(st.data_ptr()), _stream_handle(stream))
        _check(rc, "mlmc_level_paths_steps_async")
        return states, flags, st
    rc = lib().mlmc_level_paths_async(level, N, integrator, C.byref(params), seed, path_offset,
                                      C.c_void_p(states.data_ptr()), C.c_void_p(flags.data_ptr()),
                                      _stream_handle(stream))
    _check(rc, "mlmc_level_paths_async")
    return states, flags


def path_trace(level, N, integrator, params, seed, path_offset=0, stream=None):
    """Trajectories: (N, M+1, 3) fine and (N, M/2+1, 3) coarse CUDA tensors."""
    import torch
    dt = torch.float64 if params.precision == FP64 else torch.float32
    M = params.M0 << level
    tf = torch.zeros((N, M + 1, 3), dtype=dt, device="cuda")
    tc = torch.zeros((N, M // 2 + 1, 3), dtype=dt, device="cuda")
    rc = lib().mlmc_path_trace_async(level, N, integrator, C.byref(params), seed, path_offset,
                                     C.c_void_p(tf.data_ptr()), C.c_void_p(tc.data_ptr()),
                                     _stream_handle(stream))
    _check(rc, "mlmc_path_trace_async")
    return tf, tc


def path_trace_half(level, N, integrator, params, seed, path_offset=0, stream=None):
    """BAOAB's (z, w, S) after the first half of every step: (N, M, 3) fine and
    (N, M/2, 3) coarse CUDA tensors (``mlmc_path_trace_half_async``)."""
    import torch
    dt = torch.float64 if params.precision == FP64 else torch.float32
    M = params.M0 << level
    hf = torch.zeros((N, M, 3), dtype=dt, device="cuda")
    hc = torch.zeros((N, M // 2, 3), dtype=dt, device="cuda")
    rc = lib().mlmc_path_trace_half_async(level, N, integrator, C.byref(params), seed, path_offset,
                                          C.c_void_p(hf.data_ptr()), C.c_void_p(hc.data_ptr()),
                                          _stream_handle(stream))
    _check(rc, "mlmc_path_trace_half_async")
    return hf, hc


def server_query_bytes(params):
    """Bytes of the device record a query with these parameters takes in a
    server's pool (``mlmc_server_query_bytes``)."""
    return int(lib().mlmc_server_query_bytes(C.byref(params)))


class Server:
    """Continuous-batching server of dispersion queries (``mlmc_server_*``).

    ``submit`` queues a query (a ``Params`` with its own scenario and
    ``stream_id``) with its tolerance; ``tick`` takes the folded launches,
    retires the finished queries, admits queued ones whose device records
    fit, and puts one more batched launch in flight (up to four at once);
    ``poll`` returns a finished query's result and latency.  The workspace is
    sized for ``max_active`` records of 17 levels unless ``pool_bytes`` sets
    the pool explicitly.
    """

    def __init__(self, integrator=BAOAB, precision=FP32, max_active=64, seed=1, stream=None,
                 pool_bytes=None):
        import torch
        self.integrator, self.precision = integrator, precision
        if pool_bytes is None:
            nbytes = int(lib().mlmc_server_workspace_bytes(max_active))
        else:
            nbytes = int(lib().mlmc_server_workspace_bytes(0)) + int(pool_bytes)
        self._buf = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        ptr = (self._buf.data_ptr() + 255) // 256 * 256
        self.stream = stream
        self.handle = C.c_void_p()
        rc = lib().mlmc_server_create(integrator, precision, max_active, seed, C.c_void_p(ptr),
                                      nbytes, _stream_handle(stream), C.byref(self.handle))
        _check(rc, "mlmc_server_create")

    def submit(self, params, eps):
        qid = C.c_uint64()
        _check(lib().mlmc_server_submit(self.handle, C.byref(params), eps, C.byref(qid)),
               "mlmc_server_submit")
        return qid.value

    def tick(self):
        nd, na = C.c_int(), C.c_int()
        _check(lib().mlmc_server_tick(self.handle, C.byref(nd), C.byref(na)), "mlmc_server_tick")
        return nd.value, na.value

    def poll(self, qid, level_min=0):
        r = Result()
        lat = C.c_double()
        rc = lib().mlmc_server_poll(self.handle, qid, C.byref(r), C.byref(lat))
        if rc == 1:
            return None
        _check(rc, "mlmc_server_poll", allow=(ENONFINITE, ENOTCONV))
        out = _result(r, level_min)
        out["status"] = rc
        out["latency_s"] = lat.value
        return out

    def release(self, qid):
        lib().mlmc_server_release(self.handle, qid)

    def stats(self):
        o = (C.c_double * 6)()
        _check(lib().mlmc_server_stats(self.handle, o), "mlmc_server_stats")
        return dict(ticks=int(o[0]), finished=int(o[1]), path_steps=o[2], busy_s=o[3],
                    active=int(o[4]), queued=int(o[5]))

    def pool(self):
        """(record bytes in use, pool bytes)."""
        o = (C.c_uint64 * 2)()
        _check(lib().mlmc_server_pool(self.handle, o), "mlmc_server_pool")
        return int(o[0]), int(o[1])

    def run_until_idle(self, max_ticks=100000):
        for _ in range(max_ticks):
            _, left = self.tick()
            if left == 0:
                return
        raise RuntimeError("server did not drain")

    def close(self):
        if self.handle:
            lib().mlmc_server_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
