"""Python binding of the C ABI declared in include/sce.h (ctypes).

Argument marshalling only: every step runs in the CUDA library libsce.so.
Device arrays are passed as torch CUDA tensors (their data_ptr); the stream is
the tensor's current torch stream unless one is given.  A missing library is
an error -- there is no fallback.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsce.so")

CE_OK = 0
CE_ERR_INVALID_ARG = -1
CE_ERR_NOT_PSD = -2
CE_ERR_OOM = -3
CE_ERR_CUDA = -4
CE_ERR_NOT_CONVERGED = -5
CE_ERR_TIMEOUT = -6
CE_ERR_NONFINITE = -7

CE_COV_MATERN = 0
CE_COV_SEP_EXP = 1
CE_PAD_NONE = 0
CE_PAD_DOUBLING = 1
CE_PAD_SMOOTH = 2
CE_KEEP_ALL = -1
CE_KEEP_TAU_SQRT_S = -2

QOI_OUTFLOW = 0
QOI_POINT = 1
QOI_L2 = 2


class ce_cov(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nu", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("sigma2", ctypes.c_double)]


class ce_pad(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("J", ctypes.c_int), ("max_P", ctypes.c_int)]


class ce_smoothing(ctypes.Structure):
    _fields_ = [("keep_fine", ctypes.c_longlong), ("keep_coarse", ctypes.c_longlong),
                ("tie_rel_tol", ctypes.c_double)]


class ce_embedding_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("P", ctypes.c_int), ("J", ctypes.c_int),
                ("s", ctypes.c_longlong), ("keep_eff_fine", ctypes.c_longlong),
                ("keep_eff_coarse", ctypes.c_longlong), ("lambda_min", ctypes.c_double),
                ("lambda_max", ctypes.c_double), ("max_imag", ctypes.c_double)]


class darcy_problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("f", ctypes.c_double), ("rtol", ctypes.c_double),
                ("maxit", ctypes.c_int), ("precision", ctypes.c_int)]


class ce_field_task(ctypes.Structure):
    _fields_ = [("emb", ctypes.c_void_p), ("level", ctypes.c_uint32),
                ("first_sample", ctypes.c_uint64), ("count", ctypes.c_int),
                ("k_fine", ctypes.c_void_p), ("k_coarse", ctypes.c_void_p)]


class ce_levels_opts(ctypes.Structure):
    _fields_ = [("wait_cycles", ctypes.c_longlong), ("starve_task", ctypes.c_int)]


class mlmc_level_sums(ctypes.Structure):
    _fields_ = [("N", ctypes.c_longlong), ("sumY", ctypes.c_double), ("sumY2", ctypes.c_double),
                ("sumQf", ctypes.c_double), ("sumQf2", ctypes.c_double),
                ("n_failed", ctypes.c_int), ("max_iters", ctypes.c_int),
                ("total_iters", ctypes.c_longlong)]


# name -> (restype, argtypes); the exported C ABI
_P = ctypes.c_void_p
class mlmc_level_task(ctypes.Structure):
    _fields_ = [("emb", ctypes.c_void_p), ("level", ctypes.c_uint32),
                ("first_sample", ctypes.c_uint64), ("count", ctypes.c_int),
                ("Y", ctypes.c_void_p), ("qoi_f", ctypes.c_void_p), ("qoi_c", ctypes.c_void_p),
                ("sums", mlmc_level_sums), ("status", ctypes.c_int)]


class mlmc3_level_task(ctypes.Structure):
    _fields_ = [("emb", ctypes.c_void_p), ("level", ctypes.c_uint32),
                ("first_sample", ctypes.c_uint64), ("count", ctypes.c_int),
                ("Y", ctypes.c_void_p), ("sums", mlmc_level_sums), ("status", ctypes.c_int)]


class sce_server_config(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int), ("hbm_budget", ctypes.c_longlong),
                ("max_embeddings", ctypes.c_int), ("precision", ctypes.c_int),
                ("rtol", ctypes.c_double), ("maxit", ctypes.c_int),
                ("slice_vertices", ctypes.c_longlong)]


class sce_request(ctypes.Structure):
    _fields_ = [("cov", ce_cov), ("pad", ce_pad), ("n", ctypes.c_int), ("level", ctypes.c_uint32),
                ("smoothing", ctypes.c_int), ("finest", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("first_sample", ctypes.c_uint64), ("count", ctypes.c_int),
                ("qoi_index", ctypes.c_int), ("f", ctypes.c_double), ("Y", ctypes.c_void_p)]


class sce_result(ctypes.Structure):
    _fields_ = [("sums", mlmc_level_sums), ("status", ctypes.c_int), ("cache_hit", ctypes.c_int),
                ("footprint", ctypes.c_longlong), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_setup_done", ctypes.c_double),
                ("t_done", ctypes.c_double)]


class sce_server_stats_t(ctypes.Structure):
    _fields_ = [(k, ctypes.c_longlong) for k in (
        "submitted", "completed", "queued", "in_flight", "peak_in_flight", "cache_hits",
        "cache_misses", "cached", "reserved", "peak_reserved", "budget")] + [("now", ctypes.c_double)]


_SIGS = {
    "ce_setup_embedding": (ctypes.c_int, [ctypes.POINTER(ce_cov), ctypes.c_int,
                                          ctypes.POINTER(ce_pad), ctypes.POINTER(ce_smoothing),
                                          _P, ctypes.POINTER(_P),
                                          ctypes.POINTER(ce_embedding_info)]),
    "ce_get_eigenvalues": (ctypes.c_int, [_P, _P, ctypes.c_int, _P]),
    "ce_get_mask": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "ce_normals": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int,
                                  ctypes.c_longlong, ctypes.c_int, _P, _P]),
    "ce_sample_batch": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                       ctypes.c_int, ctypes.c_int, _P, _P, _P]),
    "ce_sample_batch_noalloc": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_uint32,
                                               ctypes.c_uint64, ctypes.c_int, ctypes.c_int, _P,
                                               _P, _P]),
    "darcy_solve_batch": (ctypes.c_int, [ctypes.POINTER(darcy_problem), _P, ctypes.c_int, _P, _P,
                                         _P, _P, _P]),
    "mlmc_level_estimate": (ctypes.c_int, [_P, ctypes.POINTER(darcy_problem), ctypes.c_uint64,
                                           ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int,
                                           ctypes.c_int, ctypes.POINTER(mlmc_level_sums), _P, _P,
                                           _P, _P]),
    "sce_server_create": (ctypes.c_int, [ctypes.POINTER(sce_server_config), ctypes.POINTER(_P)]),
    "sce_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(sce_request),
                                         ctypes.POINTER(ctypes.c_uint64)]),
    "sce_server_wait": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_double,
                                       ctypes.POINTER(sce_result)]),
    "sce_server_stats": (ctypes.c_int, [_P, ctypes.POINTER(sce_server_stats_t)]),
    "sce_server_destroy": (None, [_P]),
    "ce_autotune_fft": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P,
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int)]),
    "ce_qmc_setup": (ctypes.c_int, [_P, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(_P)]),
    "ce_qmc_destroy": (None, [_P]),
    "ce_sample_batch_qmc": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                           ctypes.c_uint32, ctypes.c_int, ctypes.c_int, _P, _P,
                                           _P]),
    "mlmc_level_estimate_qmc": (ctypes.c_int, [_P, ctypes.POINTER(darcy_problem),
                                               ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                               ctypes.c_uint32, ctypes.c_int, ctypes.c_int,
                                               ctypes.POINTER(mlmc_level_sums), _P, _P, _P, _P]),
    "mlmc_estimate_levels": (ctypes.c_int, [ctypes.POINTER(darcy_problem), ctypes.c_uint64,
                                            ctypes.c_int, ctypes.POINTER(mlmc_level_task),
                                            ctypes.c_int, ctypes.c_int, _P]),
    "mlmc_estimate_levels_persistent": (ctypes.c_int, [ctypes.POINTER(darcy_problem), ctypes.c_uint64,
                                            ctypes.c_int, ctypes.POINTER(mlmc_level_task),
                                            ctypes.c_int, ctypes.c_int, _P]),
    "mlmc_optimal_samples": (ctypes.c_int, [ctypes.c_int, _P, _P, ctypes.c_double, _P]),
    "mlmc_tau_exponential": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                            ctypes.POINTER(ctypes.c_double)]),
    "mlmc_tau_matern": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double,
                                       ctypes.POINTER(ctypes.c_double)]),
    "ce3_setup_embedding": (ctypes.c_int, [ctypes.POINTER(ce_cov), ctypes.c_int,
                                           ctypes.POINTER(ce_pad), ctypes.POINTER(ce_smoothing),
                                           _P, ctypes.POINTER(_P),
                                           ctypes.POINTER(ce_embedding_info)]),
    "ce3_get_info": (ctypes.c_int, [_P, ctypes.POINTER(ce_embedding_info)]),
    "ce3_get_eigenvalues": (ctypes.c_int, [_P, _P, ctypes.c_int, _P]),
    "ce3_get_mask": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "ce3_destroy": (None, [_P]),
    "ce3_sample_batch": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                        ctypes.c_int, _P, _P, _P]),
    "darcy3_solve_batch": (ctypes.c_int, [ctypes.POINTER(darcy_problem), _P, ctypes.c_int, _P,
                                          _P, _P, _P, _P]),
    "mlmc3_estimate_levels": (ctypes.c_int, [ctypes.POINTER(darcy_problem), ctypes.c_uint64,
                                             ctypes.c_int, ctypes.POINTER(mlmc3_level_task),
                                             ctypes.c_int, ctypes.c_int, _P]),
    "mlmc3_level_estimate": (ctypes.c_int, [_P, ctypes.POINTER(darcy_problem), ctypes.c_uint64,
                                            ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int,
                                            ctypes.c_int, ctypes.POINTER(mlmc_level_sums), _P,
                                            _P]),
    "ce_destroy": (None, [_P]),
    "ce_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "sce_last_error": (ctypes.c_char_p, []),
    "ce_sample_levels": (ctypes.c_int, [ctypes.POINTER(ce_field_task), ctypes.c_int,
                                        ctypes.c_uint64, ctypes.POINTER(ce_levels_opts), _P]),
    "darcy_autotune_tiles": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, _P, ctypes.POINTER(ctypes.c_int)]),
    "sce_test_fail_allocs": (None, [ctypes.c_int]),
    "darcy_solver_cache_clear": (ctypes.c_int, [_P]),
    "sce_peak_fma": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P]),
    "sce_peak_l2": (ctypes.c_int, [_P, ctypes.c_size_t, ctypes.c_int, ctypes.c_int, _P, _P]),
    "sce_profile_enable": (None, [ctypes.c_int]),
    "sce_profile_read": (ctypes.c_int, [ctypes.c_int, _P, _P, _P]),
    "sce_profile_count": (ctypes.c_int, []),
    "sce_profile_name": (ctypes.c_char_p, [ctypes.c_int]),
}
EXPORTED = tuple(_SIGS)

_lib = None


class SceError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        detail = ""
        if status in (CE_ERR_CUDA, CE_ERR_OOM, CE_ERR_INVALID_ARG) and _lib is not None:
            text = _lib.sce_last_error()
            detail = f" [{text.decode(errors='replace')}]" if text else ""
        super().__init__(f"{what}: {status_string(status)} ({status}){detail}")


def load(path=None):
    """Loads libsce.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libsce.so not built at {p}: run paper_2306_13493_gb300.build")
    lib = ctypes.CDLL(p)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def status_string(status):
    return load().ce_status_string(int(status)).decode()


def last_error():
    return load().sce_last_error().decode()


def _check(status, what, allow=()):
    if status != CE_OK and status not in allow:
        raise SceError(status, what)
    return status


def _stream(stream, tensor=None):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    import torch
    dev = tensor.device if tensor is not None and tensor.is_cuda else None
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


class Embedding:
    """Owner of a ce_embedding_t handle (destroyed with the object)."""

    def __init__(self, handle, info):
        self.handle = handle
        self.info = info

    @property
    def n(self):
        return self.info.n

    @property
    def P(self):
        return self.info.P

    def close(self):
        if self.handle:
            load().ce_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ce_setup_embedding(kind, nu, lam, sigma2, n, pad_mode=CE_PAD_DOUBLING, J=-1, max_P=8192,
                       keep_fine=-1, keep_coarse=-1, tie_rel_tol=1e-10, stream=None):
    lib = load()
    cov = ce_cov(kind, nu, lam, sigma2)
    pad = ce_pad(pad_mode, J, max_P)
    sm = ce_smoothing(keep_fine, keep_coarse, tie_rel_tol)
    h = ctypes.c_void_p()
    info = ce_embedding_info()
    _check(lib.ce_setup_embedding(ctypes.byref(cov), n, ctypes.byref(pad), ctypes.byref(sm),
                                  _stream(stream), ctypes.byref(h), ctypes.byref(info)),
           "ce_setup_embedding")
    return Embedding(h, info)


def ce_get_eigenvalues(emb, out, stream=None):
    """out: torch float64 tensor of P*P elements (device or host)."""
    _check(load().ce_get_eigenvalues(emb.handle, _ptr(out), int(out.is_cuda), _stream(stream, out)),
           "ce_get_eigenvalues")
    return out


def ce_get_mask(emb, which, out):
    """out: contiguous host uint8 tensor/array of P*P elements."""
    ptr = out.ctypes.data if hasattr(out, "ctypes") else out.data_ptr()
    _check(load().ce_get_mask(emb.handle, which, ctypes.c_void_p(ptr)), "ce_get_mask")
    return out


def ce_normals(seed, level, first_sample, count, length, precision, out, stream=None):
    _check(load().ce_normals(seed, level, first_sample, count, length, precision, _ptr(out),
                             _stream(stream, out)), "ce_normals")
    return out


def ce_sample_batch(emb, seed, level, first_sample, count, precision, k_fine=None,
                    k_coarse=None, stream=None):
    t = k_fine if k_fine is not None else k_coarse
    _check(load().ce_sample_batch(emb.handle, seed, level, first_sample, count, precision,
                                  _ptr(k_fine), _ptr(k_coarse), _stream(stream, t)),
           "ce_sample_batch")


def ce_sample_batch_noalloc(emb, seed, level, first_sample, count, precision, k_fine,
                            k_coarse=None, stream=None):
    """ce_sample_batch without any device allocation (fixed internal scratch)."""
    _check(load().ce_sample_batch_noalloc(emb.handle, seed, level, first_sample, count,
                                          precision, _ptr(k_fine), _ptr(k_coarse),
                                          _stream(stream, k_fine)), "ce_sample_batch_noalloc")


def darcy_solve_batch(n, k, count, qoi, f=0.0, rtol=1e-10, maxit=1000, precision=32, iters=None,
                      status=None, u_out=None, stream=None, allow_not_converged=False):
    prob = darcy_problem(n, f, rtol, maxit, precision)
    allow = (CE_ERR_NOT_CONVERGED,) if allow_not_converged else ()
    return _check(load().darcy_solve_batch(ctypes.byref(prob), _ptr(k), count, _ptr(qoi),
                                           _ptr(iters), _ptr(status), _ptr(u_out),
                                           _stream(stream, k)), "darcy_solve_batch", allow)


def mlmc_level_estimate(emb, seed, level, first_sample, count, qoi_index=QOI_OUTFLOW, f=0.0,
                        rtol=1e-10, maxit=1000, precision=32, Y=None, qoi_f=None, qoi_c=None,
                        stream=None, allow_not_converged=False):
    prob = darcy_problem(emb.n, f, rtol, maxit, precision)
    out = mlmc_level_sums()
    allow = (CE_ERR_NOT_CONVERGED,) if allow_not_converged else ()
    st = _check(load().mlmc_level_estimate(emb.handle, ctypes.byref(prob), seed, level,
                                           first_sample, count, qoi_index, ctypes.byref(out),
                                           _ptr(Y), _ptr(qoi_f), _ptr(qoi_c), _stream(stream, Y)),
                "mlmc_level_estimate", allow)
    return out, st


def mlmc_estimate_levels(tasks, seed, qoi_index=QOI_OUTFLOW, f=0.0, rtol=1e-10, maxit=1000,
                         precision=32, max_concurrency=8, stream=None, allow_not_converged=False,
                         persistent=False):
    """All levels of one MLMC step in one call.  ``tasks``: sequence of dicts
    with keys emb, level, first_sample, count and optionally Y, qoi_f, qoi_c
    (CUDA tensors).  persistent=True: every level's fields in one persistent
    launch first (mlmc_estimate_levels_persistent).  Returns
    ([mlmc_level_sums per task], [status per task], overall status)."""
    if not tasks:
        return [], [], CE_OK
    arr = (mlmc_level_task * len(tasks))()
    for t, d in zip(arr, tasks):
        h = d["emb"].handle
        t.emb = h.value if isinstance(h, ctypes.c_void_p) else h
        t.level = d["level"]
        t.first_sample = d["first_sample"]
        t.count = d["count"]
        t.Y, t.qoi_f, t.qoi_c = (_ptr(d.get(k)).value for k in ("Y", "qoi_f", "qoi_c"))
    prob = darcy_problem(tasks[0]["emb"].n, f, rtol, maxit, precision)
    allow = (CE_ERR_NOT_CONVERGED,) if allow_not_converged else ()
    ref = next((d[k] for d in tasks for k in ("Y", "qoi_f", "qoi_c") if d.get(k) is not None),
               None)
    fn = load().mlmc_estimate_levels_persistent if persistent else load().mlmc_estimate_levels
    st = _check(fn(ctypes.byref(prob), seed, qoi_index, arr, len(tasks), max_concurrency,
                   _stream(stream, ref)),
                "mlmc_estimate_levels_persistent" if persistent else "mlmc_estimate_levels", allow)
    return [mlmc_level_sums.from_buffer_copy(t.sums) for t in arr], [t.status for t in arr], st


class Server:
    """Request server of the C ABI (sce_server_*): submit MLMC level requests,
    wait for their results.  Requests are dicts with keys kind, nu, lam,
    sigma2, n, level, count and optionally pad_mode (2), J (-1), max_P (8192),
    smoothing (1), finest (0), seed (0), first_sample (0), qoi_index (1), f (1.0),
    Y (CUDA tensor of count doubles)."""

    def __init__(self, slots=8, hbm_budget=0, max_embeddings=256, precision=32, rtol=1e-10,
                 maxit=2000, slice_vertices=0):
        self._lib = load()
        cfg = sce_server_config(slots, hbm_budget, max_embeddings, precision, rtol, maxit,
                                slice_vertices)
        h = _P()
        _check(self._lib.sce_server_create(ctypes.byref(cfg), ctypes.byref(h)), "sce_server_create")
        self.handle = h
        self._keep = {}

    def submit(self, req):
        r = sce_request()
        r.cov = ce_cov(req.get("kind", CE_COV_MATERN), req.get("nu", 0.5), req["lam"],
                       req.get("sigma2", 1.0))
        r.pad = ce_pad(req.get("pad_mode", CE_PAD_SMOOTH), req.get("J", -1),
                       req.get("max_P", 8192))
        r.n, r.level, r.count = req["n"], req["level"], req["count"]
        r.smoothing, r.finest = req.get("smoothing", 1), req.get("finest", 0)
        r.seed, r.first_sample = req.get("seed", 0), req.get("first_sample", 0)
        r.qoi_index, r.f = req.get("qoi_index", QOI_POINT), req.get("f", 1.0)
        r.Y = _ptr(req.get("Y")).value
        t = ctypes.c_uint64()
        _check(self._lib.sce_server_submit(self.handle, ctypes.byref(r), ctypes.byref(t)),
               "sce_server_submit")
        if req.get("Y") is not None:
            self._keep[t.value] = req["Y"]
        return t.value

    def wait(self, ticket, timeout=-1.0):
        """The sce_result of `ticket`, or None if not done within `timeout` s."""
        res = sce_result()
        st = self._lib.sce_server_wait(self.handle, ticket, timeout, ctypes.byref(res))
        if st == CE_ERR_TIMEOUT:
            return None
        _check(st, "sce_server_wait")
        self._keep.pop(ticket, None)
        return res

    def stats(self):
        s = sce_server_stats_t()
        _check(self._lib.sce_server_stats(self.handle, ctypes.byref(s)), "sce_server_stats")
        return {k: getattr(s, k) for k, _ in s._fields_}

    def close(self):
        if self.handle:
            self._lib.sce_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def ce_autotune_fft(emb, precision=32, count=32, reps=3, stream=None):
    """Tunes the FFT launch shapes for emb's P; returns {"row": (tpf, F), "col": (tpf, F)}."""
    v = [ctypes.c_int() for _ in range(4)]
    _check(load().ce_autotune_fft(emb.handle, precision, count, reps, _stream(stream),
                                  *[ctypes.byref(x) for x in v]), "ce_autotune_fft")
    return {"row": (v[0].value, v[1].value), "col": (v[2].value, v[3].value)}


def ce_sample_levels(tasks, seed, wait_cycles=0, starve_task=-1, stream=None):
    """Fields of several levels in one persistent launch (FP32).  ``tasks``:
    dicts with emb, level, first_sample, count, k_fine and optionally
    k_coarse (CUDA float tensors).  Synchronises the stream."""
    arr = (ce_field_task * len(tasks))()
    for t, d in zip(arr, tasks):
        h = d["emb"].handle
        t.emb = h.value if isinstance(h, ctypes.c_void_p) else h
        t.level = d["level"]
        t.first_sample = d["first_sample"]
        t.count = d["count"]
        t.k_fine = d["k_fine"].data_ptr()
        t.k_coarse = d["k_coarse"].data_ptr() if d.get("k_coarse") is not None else None
    opts = ce_levels_opts(wait_cycles, starve_task)
    _check(load().ce_sample_levels(arr, len(tasks), seed, ctypes.byref(opts),
                                   _stream(stream, tasks[0]["k_fine"])), "ce_sample_levels")


def darcy_autotune_tiles(n, precision=32, count=64, reps=3, stream=None):
    """Tunes the multigrid window height for n-cell grids; returns the height."""
    h = ctypes.c_int()
    _check(load().darcy_autotune_tiles(n, precision, count, reps, _stream(stream),
                                       ctypes.byref(h)), "darcy_autotune_tiles")
    return h.value


class QmcLattice:
    """Lattice table of the quasi-Monte Carlo sampler (ce_qmc_setup) for an
    Embedding: N points (a power of two), Korobov parameter a (odd)."""

    def __init__(self, emb, N, a):
        h = _P()
        _check(load().ce_qmc_setup(emb.handle, N, a, ctypes.byref(h)), "ce_qmc_setup")
        self.handle, self.emb, self.N, self.a = h, emb, N, a

    def close(self):
        if self.handle:
            load().ce_qmc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ce_sample_batch_qmc(q, seed, level, shift, first_point, count, precision, k_fine=None,
                        k_coarse=None, stream=None):
    t = k_fine if k_fine is not None else k_coarse
    _check(load().ce_sample_batch_qmc(q.handle, seed, level, shift, first_point, count, precision,
                                      _ptr(k_fine), _ptr(k_coarse), _stream(stream, t)),
           "ce_sample_batch_qmc")


def mlmc_level_estimate_qmc(q, seed, level, shift, first_point, count, qoi_index=QOI_OUTFLOW,
                            f=0.0, rtol=1e-10, maxit=1000, precision=32, Y=None, qoi_f=None,
                            qoi_c=None, stream=None, allow_not_converged=False):
    prob = darcy_problem(q.emb.n, f, rtol, maxit, precision)
    out = mlmc_level_sums()
    allow = (CE_ERR_NOT_CONVERGED,) if allow_not_converged else ()
    st = _check(load().mlmc_level_estimate_qmc(q.handle, ctypes.byref(prob), seed, level, shift,
                                               first_point, count, qoi_index, ctypes.byref(out),
                                               _ptr(Y), _ptr(qoi_f), _ptr(qoi_c),
                                               _stream(stream, Y)),
                "mlmc_level_estimate_qmc", allow)
    return out, st


class Embedding3(Embedding):
    """Owner of a ce3_embedding_t handle (three-dimensional grids)."""

    def close(self):
        if self.handle:
            load().ce3_destroy(self.handle)
            self.handle = None


def ce3_setup_embedding(kind, nu, lam, sigma2, n, pad_mode=CE_PAD_DOUBLING, J=-1, max_P=512,
                        keep_fine=-1, keep_coarse=-1, tie_rel_tol=1e-10, stream=None):
    lib = load()
    cov = ce_cov(kind, nu, lam, sigma2)
    pad = ce_pad(pad_mode, J, max_P)
    sm = ce_smoothing(keep_fine, keep_coarse, tie_rel_tol)
    h = ctypes.c_void_p()
    info = ce_embedding_info()
    _check(lib.ce3_setup_embedding(ctypes.byref(cov), n, ctypes.byref(pad), ctypes.byref(sm),
                                   _stream(stream), ctypes.byref(h), ctypes.byref(info)),
           "ce3_setup_embedding")
    return Embedding3(h, info)


def ce3_get_eigenvalues(emb, out, stream=None):
    """out: torch float64 tensor of P^3 elements (device or host)."""
    _check(load().ce3_get_eigenvalues(emb.handle, _ptr(out), int(out.is_cuda),
                                      _stream(stream, out)), "ce3_get_eigenvalues")
    return out


def ce3_get_mask(emb, which, out):
    """out: contiguous host uint8 array/tensor of P^3 elements."""
    ptr = out.ctypes.data if hasattr(out, "ctypes") else out.data_ptr()
    _check(load().ce3_get_mask(emb.handle, which, ctypes.c_void_p(ptr)), "ce3_get_mask")
    return out


def ce3_sample_batch(emb, seed, level, first_sample, count, k_fine=None, k_coarse=None,
                     stream=None):
    """FP32 fields: k_fine (count*(n+1)^3), k_coarse (count*(n/2+1)^3), torch float32 on the device."""
    t = k_fine if k_fine is not None else k_coarse
    _check(load().ce3_sample_batch(emb.handle, seed, level, first_sample, count, _ptr(k_fine),
                                   _ptr(k_coarse), _stream(stream, t)), "ce3_sample_batch")


def darcy3_solve_batch(n, k, count, qoi, f=0.0, rtol=1e-10, maxit=1000, iters=None, status=None,
                       u_out=None, stream=None, allow_not_converged=False):
    prob = darcy_problem(n, f, rtol, maxit, 32)
    allow = (CE_ERR_NOT_CONVERGED,) if allow_not_converged else ()
    return _check(load().darcy3_solve_batch(ctypes.byref(prob), _ptr(k), count, _ptr(qoi),
                                            _ptr(iters), _ptr(status), _ptr(u_out),
                                            _stream(stream, k)), "darcy3_solve_batch", allow)


def mlmc3_level_estimate(emb, seed, level, first_sample, count, qoi_index=QOI_OUTFLOW, f=0.0,
                         rtol=1e-10, maxit=1000, Y=None, stream=None, allow_not_converged=False):
    prob = darcy_problem(emb.n, f, rtol, maxit, 32)
    out = mlmc_level_sums()
    allow = (CE_ERR_NOT_CONVERGED,) if allow_not_converged else ()
    st = _check(load().mlmc3_level_estimate(emb.handle, ctypes.byref(prob), seed, level,
                                            first_sample, count, qoi_index, ctypes.byref(out),
                                            _ptr(Y), _stream(stream, Y)),
                "mlmc3_level_estimate", allow)
    return out, st


def mlmc3_estimate_levels(tasks, seed, qoi_index=QOI_OUTFLOW, f=0.0, rtol=1e-10, maxit=1000,
                          max_concurrency=8, stream=None, allow_not_converged=False):
    """All levels of one d = 3 MLMC step in one call.  ``tasks``: sequence of
    dicts with keys emb (Embedding3), level, first_sample, count and optionally
    Y (CUDA tensor).  Returns ([mlmc_level_sums per task], [status per task],
    overall status)."""
    if not tasks:
        return [], [], CE_OK
    arr = (mlmc3_level_task * len(tasks))()
    for t, d in zip(arr, tasks):
        h = d["emb"].handle
        t.emb = h.value if isinstance(h, ctypes.c_void_p) else h
        t.level = d["level"]
        t.first_sample = d["first_sample"]
        t.count = d["count"]
        t.Y = _ptr(d.get("Y")).value
    prob = darcy_problem(tasks[0]["emb"].n, f, rtol, maxit, 32)
    allow = (CE_ERR_NOT_CONVERGED,) if allow_not_converged else ()
    ref = next((d["Y"] for d in tasks if d.get("Y") is not None), None)
    st = _check(load().mlmc3_estimate_levels(ctypes.byref(prob), seed, qoi_index, arr,
                                             len(tasks), max_concurrency, _stream(stream, ref)),
                "mlmc3_estimate_levels", allow)
    return [mlmc_level_sums.from_buffer_copy(t.sums) for t in arr], [t.status for t in arr], st


def sce_profile_enable(on):
    load().sce_profile_enable(int(bool(on)))


def sce_profile_read():
    """{family name: (ms, algorithmic bytes, launches)} for families that ran."""
    lib = load()
    out = {}
    for i in range(lib.sce_profile_count()):
        ms, by, nl = ctypes.c_double(), ctypes.c_double(), ctypes.c_longlong()
        _check(lib.sce_profile_read(i, ctypes.byref(ms), ctypes.byref(by), ctypes.byref(nl)),
               "sce_profile_read")
        if nl.value:
            out[lib.sce_profile_name(i).decode()] = (ms.value, by.value, nl.value)
    return out


def mlmc_optimal_samples(V, C, eps):
    import numpy as np
    V = np.ascontiguousarray(V, dtype=np.float64)
    C = np.ascontiguousarray(C, dtype=np.float64)
    N = np.zeros(len(V), dtype=np.int64)
    _check(load().mlmc_optimal_samples(len(V), ctypes.c_void_p(V.ctypes.data),
                                       ctypes.c_void_p(C.ctypes.data), eps,
                                       ctypes.c_void_p(N.ctypes.data)), "mlmc_optimal_samples")
    return N


def mlmc_tau_exponential(s, alpha, cs_over_calpha=1.0):
    t = ctypes.c_double()
    _check(load().mlmc_tau_exponential(float(s), float(alpha), float(cs_over_calpha),
                                       ctypes.byref(t)), "mlmc_tau_exponential")
    return t.value


def mlmc_tau_matern(h, J, nu, alpha, cs_over_calpha=1.0):
    t = ctypes.c_double()
    _check(load().mlmc_tau_matern(float(h), float(J), float(nu), float(alpha),
                                  float(cs_over_calpha), ctypes.byref(t)), "mlmc_tau_matern")
    return t.value


def sce_peak_fma(out, blocks, iters, stream=None):
    """Launches the FP32 FMA issue-rate kernel (blocks * 8 * iters * 128 FMA
    warp instructions); the caller times it on ``stream``."""
    _check(load().sce_peak_fma(_ptr(out), blocks, iters, _stream(stream, out)), "sce_peak_fma")


def sce_peak_l2(buf, reps, blocks, out, stream=None):
    """Launches the L2 read-bandwidth kernel over the CUDA tensor ``buf``
    (buf.nbytes * reps bytes); the caller times it on ``stream``."""
    nbytes = buf.numel() * buf.element_size()
    _check(load().sce_peak_l2(_ptr(buf), nbytes, reps, blocks, _ptr(out), _stream(stream, out)),
           "sce_peak_l2")


def sce_test_fail_allocs(count):
    """Test hook: the next `count` library allocations fail with CE_ERR_OOM."""
    load().sce_test_fail_allocs(int(count))


def darcy_solver_cache_clear(stream=None):
    """Frees the idle solvers (and their graphs) kept under SCE_GRAPHS=1."""
    _check(load().darcy_solver_cache_clear(_stream(stream)), "darcy_solver_cache_clear")
