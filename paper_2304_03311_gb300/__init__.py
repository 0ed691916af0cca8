"""GB300 (sm_103a) library for the Jarzynski replica-gluing estimator of
Renyi-2 entanglement entropy increments and the entropic c-function
(Bulgarelli & Panero, arXiv:2304.03311).

This module is a thin ctypes binding of the C ABI declared in
``include/isingjz.h``: same names, same arguments, marshalling only.  Every step
of the method runs in the CUDA kernels of ``libisingjz.so``; there is no CPU
fallback, and importing the binding fails loudly when the library is missing.

Buffers may be torch tensors (CUDA or CPU) or numpy arrays; the library
decides from the pointer whether it writes device memory directly (the call
then only enqueues work; use ``ising_sync``) or copies back to host memory.
"""
from __future__ import annotations

import ctypes
import os

from .build import LIB as _LIB_PATH
from .build import LIB_DEBUG as _LIB_DEBUG_PATH

__all__ = [
    "IsingError", "JzParams", "lib_path", "load", "ising_replica_init", "ising_replica_free",
    "ising_sync", "jarzynski_run", "jarzynski_run_ex", "jarzynski_run_batch", "jarzynski_run_plain",
    "estimator_reduce", "ising_strerror", "jz_params_default", "ising_probe",
    "jarzynski_run_noalloc", "ising_binary_version", "ising_cancel", "ising_cancel_reset",
    "jarzynski_run_resumable", "jz_cancel", "jz_server_set_log", "jz_result_json", "TuneCache",
    "ising_autotune_cached", "ising_bounds_status", "use_debug_library", "ising_launch_shape",
]

ISING_OK = 0
ISING_ERR_ARG = -1
ISING_ERR_ODD_EXTENT = -2
ISING_ERR_L_RANGE = -3
ISING_ERR_NOMEM = -4
ISING_ERR_CUDA = -5
ISING_ERR_TIMEOUT = -6
ISING_ERR_UNSUPPORTED = -7
ISING_ERR_NOT_FOUND = -8
ISING_ERR_PENDING = -9
ISING_ERR_SCRATCH_LIMIT = -10
ISING_ERR_CANCELLED = -11


class JzParams(ctypes.Structure):
    """Mirror of ``jz_params`` in include/isingjz.h."""
    _fields_ = [
        ("d", ctypes.c_int), ("L", ctypes.c_int), ("L_t", ctypes.c_int),
        ("update", ctypes.c_int), ("beta", ctypes.c_double), ("l", ctypes.c_int),
        ("n_step", ctypes.c_int), ("n_sweep", ctypes.c_int), ("n_therm", ctypes.c_int),
        ("n_traj", ctypes.c_int), ("direction", ctypes.c_int),
        ("traj0", ctypes.c_longlong), ("seed", ctypes.c_uint64), ("protocol", ctypes.c_int),
        ("n_replica", ctypes.c_int), ("whole", ctypes.c_int), ("therm_update", ctypes.c_int),
    ]


class JzResult(ctypes.Structure):
    """Mirror of ``jz_result`` in include/isingjz.h."""
    _fields_ = [
        ("status", ctypes.c_int), ("log_ratio", ctypes.c_double), ("delta_S2", ctypes.c_double),
        ("delta_S2_err", ctypes.c_double), ("submit_s", ctypes.c_double),
        ("start_s", ctypes.c_double), ("done_s", ctypes.c_double), ("updates", ctypes.c_longlong),
    ]


class IsingError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {ising_strerror(code)} ({code})")


_lib = None


def lib_path() -> str:
    return _LIB_PATH


def use_debug_library() -> None:
    """Bind to the bounds-checked build libisingjz_debug.so (build it with
    ``build.build(debug=True)``) instead of the release library.  Must be
    called before the first call into the library in this process."""
    global _LIB_PATH
    if _lib is not None:
        raise RuntimeError("the release library is already loaded in this process")
    _LIB_PATH = _LIB_DEBUG_PATH


def load():
    """Load libisingjz.so (build it with ``paper_2304_03311_gb300.build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is missing: run paper_2304_03311_gb300.build.build() "
                          "(nvcc, sm_103a) before using the library")
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    sig = {
        "jz_params_default": (ctypes.c_int, [P(JzParams)]),
        "ising_replica_init": (ctypes.c_int, [P(vp), ctypes.c_int, ctypes.c_size_t, vp]),
        "ising_replica_free": (None, [vp]),
        "ising_sync": (ctypes.c_int, [vp]),
        "ising_last_launch_ms": (ctypes.c_int, [vp, P(ctypes.c_float)]),
        "jarzynski_run": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_uint64, vp]),
        "jarzynski_run_ex": (ctypes.c_int, [vp, P(JzParams), vp, vp]),
        "jarzynski_run_segment": (ctypes.c_int, [vp, P(JzParams), ctypes.c_int, ctypes.c_int,
                                                 vp, vp]),
        "jarzynski_run_batch": (ctypes.c_int, [vp, P(JzParams), ctypes.c_int, P(vp)]),
        "jarzynski_run_plain": (ctypes.c_int, [vp, P(JzParams), vp, vp]),
        "jarzynski_run_noalloc": (ctypes.c_int, [P(JzParams), vp, vp]),
        "estimator_reduce": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int, P(ctypes.c_double),
                                            P(ctypes.c_double), P(ctypes.c_double)]),
        "ising_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "ising_probe": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, P(ctypes.c_double)]),
        "ising_binary_version": (ctypes.c_int, [ctypes.c_int, P(ctypes.c_int)]),
        "ising_bounds_status": (ctypes.c_int, [P(ctypes.c_uint), P(ctypes.c_uint), ctypes.c_int]),
        "ising_cancel": (ctypes.c_int, [vp]),
        "ising_cancel_reset": (ctypes.c_int, [vp]),
        "jarzynski_run_resumable": (ctypes.c_int, [vp, P(JzParams), ctypes.c_int, ctypes.c_int,
                                                   P(ctypes.c_int), vp, vp]),
        "jz_cancel": (ctypes.c_int, [vp, ctypes.c_uint64]),
        "jz_server_set_log": (ctypes.c_int, [vp, ctypes.c_char_p]),
        "jz_result_json": (ctypes.c_int, [ctypes.c_uint64, P(JzParams), P(JzResult),
                                          ctypes.c_char_p, ctypes.c_size_t]),
        "jz_tune_cache_create": (ctypes.c_int, [P(vp)]),
        "jz_tune_cache_free": (None, [vp]),
        "jz_tune_cache_load": (ctypes.c_int, [vp, ctypes.c_char_p]),
        "jz_tune_cache_save": (ctypes.c_int, [vp, ctypes.c_char_p]),
        "jz_tune_cache_put": (ctypes.c_int, [vp, ctypes.c_char_p, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int]),
        "jz_tune_cache_get": (ctypes.c_int, [vp, ctypes.c_char_p, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             P(ctypes.c_int)]),
        "jz_tune_cache_size": (ctypes.c_int, [vp, P(ctypes.c_int)]),
        "ising_autotune_cached": (ctypes.c_int, [vp, vp, P(JzParams), P(ctypes.c_int),
                                                 P(ctypes.c_int)]),
        "ising_set_threads": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int]),
        "ising_autotune": (ctypes.c_int, [vp, P(JzParams), P(ctypes.c_int)]),
        "ising_launch_shape": (ctypes.c_int, [vp, P(JzParams), P(ctypes.c_int)]),
        "jz_plan_create": (ctypes.c_int, [vp, P(JzParams), ctypes.c_int, P(vp), vp, ctypes.c_int,
                                          P(vp)]),
        "jz_plan_launch": (ctypes.c_int, [vp]),
        "jz_plan_info": (ctypes.c_int, [vp, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int)]),
        "jz_plan_free": (None, [vp]),
        "jz_server_create": (ctypes.c_int, [vp, ctypes.c_size_t, ctypes.c_int, P(vp)]),
        "jz_submit": (ctypes.c_int, [vp, P(JzParams), P(ctypes.c_uint64)]),
        "jz_poll": (ctypes.c_int, [vp, ctypes.c_uint64, P(JzResult)]),
        "jz_wait": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.c_double, P(JzResult)]),
        "jz_server_work": (ctypes.c_int, [vp, ctypes.c_uint64, vp]),
        "jz_server_free": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(buf):
    """Raw address of a torch tensor or numpy array (None passes NULL)."""
    if buf is None:
        return None
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            raise ValueError("buffer must be contiguous")
        return buf.data_ptr()
    if hasattr(buf, "ctypes"):
        if not buf.flags["C_CONTIGUOUS"] or not buf.flags["WRITEABLE"]:
            raise ValueError("buffer must be contiguous and writeable")
        return buf.ctypes.data
    raise TypeError(f"unsupported buffer type {type(buf)!r}")


def _check(code: int, where: str):
    if code != ISING_OK:
        raise IsingError(code, where)


def ising_strerror(code: int) -> str:
    return load().ising_strerror(int(code)).decode()


def jz_params_default() -> JzParams:
    p = JzParams()
    _check(load().jz_params_default(ctypes.byref(p)), "jz_params_default")
    return p


def ising_replica_init(device: int = 0, hbm_budget_bytes: int = 0, cuda_stream: int | None = None):
    """Returns an opaque context handle (int).  cuda_stream: a cudaStream_t as
    an integer (e.g. ``torch.cuda.current_stream().cuda_stream``) or None."""
    ctx = ctypes.c_void_p()
    _check(load().ising_replica_init(ctypes.byref(ctx), int(device), int(hbm_budget_bytes),
                                     cuda_stream), "ising_replica_init")
    return ctx.value


def ising_replica_free(ctx) -> None:
    load().ising_replica_free(ctx)


def ising_sync(ctx) -> None:
    _check(load().ising_sync(ctx), "ising_sync")


def ising_last_launch_ms(ctx) -> float:
    """Device time (ms) of the last run call's kernel launches, copies excluded."""
    ms = ctypes.c_float()
    _check(load().ising_last_launch_ms(ctx, ctypes.byref(ms)), "ising_last_launch_ms")
    return ms.value


def jarzynski_run(ctx, d, L, L_t, beta, l, n_step, n_sweep, n_traj, seed, work_int_out):
    _check(load().jarzynski_run(ctx, int(d), int(L), int(L_t), float(beta), int(l), int(n_step),
                                int(n_sweep), int(n_traj), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                _ptr(work_int_out)), "jarzynski_run")


METROPOLIS, SWENDSEN_WANG = 0, 1
SW_THERM = 1   # jz_params.therm_update: Swendsen-Wang thermalisation


def make_params(d, L, L_t, beta, l, n_step, n_sweep, n_traj, seed=0, *, n_therm=1000,
                direction=1, traj0=0, update=METROPOLIS, protocol=1, n_replica=2,
                whole=False, therm_update=0) -> JzParams:
    """therm_update=SW_THERM thermalises with Swendsen-Wang clusters before a
    Metropolis protocol (see include/isingjz.h)."""
    p = jz_params_default()
    p.update = int(update)
    p.therm_update = int(therm_update)
    p.protocol = int(protocol)
    p.n_replica = int(n_replica)
    p.whole = int(bool(whole))
    p.d, p.L, p.L_t, p.beta, p.l = int(d), int(L), int(L_t), float(beta), int(l)
    p.n_step, p.n_sweep, p.n_traj = int(n_step), int(n_sweep), int(n_traj)
    p.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    p.n_therm, p.direction, p.traj0 = int(n_therm), int(direction), int(traj0)
    return p


def jarzynski_run_ex(ctx, params: JzParams, work_int_out, spins_out=None):
    _check(load().jarzynski_run_ex(ctx, ctypes.byref(params), _ptr(work_int_out),
                                   _ptr(spins_out)), "jarzynski_run_ex")


def jarzynski_run_segment(ctx, params: JzParams, k_begin: int, k_end: int, work_io, spins_io):
    """Protocol steps k_begin..k_end-1 resumed from device buffers work_io and
    spins_io (see include/isingjz.h); both are updated in place."""
    _check(load().jarzynski_run_segment(ctx, ctypes.byref(params), int(k_begin), int(k_end),
                                        _ptr(work_io), _ptr(spins_io)), "jarzynski_run_segment")


def jarzynski_run_plain(ctx, params: JzParams, work_int_out, spins_out=None):
    _check(load().jarzynski_run_plain(ctx, ctypes.byref(params), _ptr(work_int_out),
                                      _ptr(spins_out)), "jarzynski_run_plain")


def jarzynski_run_noalloc(params: JzParams, work_int_out, cuda_stream: int | None = None):
    """The allocation-free entry point (see include/isingjz.h): work_int_out
    must be device memory; returns once the work is enqueued on cuda_stream."""
    _check(load().jarzynski_run_noalloc(ctypes.byref(params), _ptr(work_int_out), cuda_stream),
           "jarzynski_run_noalloc")


def jarzynski_run_batch(ctx, params_list, work_outs):
    n = len(params_list)
    arr = (JzParams * n)(*params_list)
    outs = (ctypes.c_void_p * n)(*[_ptr(w) for w in work_outs])
    _check(load().jarzynski_run_batch(ctx, arr, n, outs), "jarzynski_run_batch")


def estimator_reduce(ctx, work_int, n_traj, beta, n_step, direction=1, n_jack_bins=32):
    """Returns (ln <e^-W>, Delta S_2, jackknife error of Delta S_2)."""
    lr, ds, err = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().estimator_reduce(ctx, _ptr(work_int), int(n_traj), float(beta), int(n_step),
                                   int(direction), int(n_jack_bins), ctypes.byref(lr),
                                   ctypes.byref(ds), ctypes.byref(err)), "estimator_reduce")
    return lr.value, ds.value, err.value


def ising_probe(device: int, kind: int) -> float:
    """Integer-issue probe rate (see include/isingjz.h): kinds 0-2 in
    thread-instructions/s, kind 3 in Philox4x32-10 blocks/s."""
    r = ctypes.c_double()
    _check(load().ising_probe(int(device), int(kind), ctypes.byref(r)), "ising_probe")
    return r.value


def ising_binary_version(device: int = 0) -> int:
    """Compute capability the device code was built for (103 = sm_103a)."""
    v = ctypes.c_int()
    _check(load().ising_binary_version(int(device), ctypes.byref(v)), "ising_binary_version")
    return v.value


def ising_set_threads(ctx, d: int, L: int, L_t: int, threads: int) -> None:
    """Fix the CTA size for lattices of shape (d, L, L_t) (0 = default)."""
    _check(load().ising_set_threads(ctx, int(d), int(L), int(L_t), int(threads)),
           "ising_set_threads")


def ising_launch_shape(ctx, params: JzParams) -> dict:
    """The launch shape jarzynski_run_ex would use for `params` in this context."""
    v = (ctypes.c_int * 5)()
    _check(load().ising_launch_shape(ctx, ctypes.byref(params), v), "ising_launch_shape")
    return {"team_threads": v[0], "teams": v[1], "cta_threads": v[2], "warp": bool(v[3]),
            "hbm": bool(v[4])}


def ising_autotune(ctx, params: JzParams) -> int:
    """Time the admissible CTA sizes and the default shape on a short sample of
    `params`, keep the fastest for its shape in the context, and return its
    CTA size (0 when the default shape won)."""
    t = ctypes.c_int()
    _check(load().ising_autotune(ctx, ctypes.byref(params), ctypes.byref(t)), "ising_autotune")
    return t.value


def jz_plan_create(ctx, params_list, work_outs, est_out=None, cta_threads: int = 0):
    """Persistent-launch plan for an uneven batch (see include/isingjz.h);
    work_outs and est_out must be device memory.  Returns the plan handle."""
    n = len(params_list)
    arr = (JzParams * n)(*params_list)
    outs = (ctypes.c_void_p * n)(*[_ptr(w) for w in work_outs])
    plan = ctypes.c_void_p()
    _check(load().jz_plan_create(ctx, arr, n, outs, _ptr(est_out), int(cta_threads),
                                 ctypes.byref(plan)), "jz_plan_create")
    return plan.value


def jz_plan_launch(plan) -> None:
    _check(load().jz_plan_launch(plan), "jz_plan_launch")


def jz_plan_info(plan):
    """(CTA size, grid size, work items) of a plan."""
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().jz_plan_info(plan, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "jz_plan_info")
    return a.value, b.value, c.value


def jz_plan_free(plan) -> None:
    load().jz_plan_free(plan)


def jz_server_create(ctx, hbm_budget_bytes: int, max_inflight: int):
    s = ctypes.c_void_p()
    _check(load().jz_server_create(ctx, int(hbm_budget_bytes), int(max_inflight),
                                   ctypes.byref(s)), "jz_server_create")
    return s.value


def jz_submit(server, params: JzParams) -> int:
    jid = ctypes.c_uint64()
    _check(load().jz_submit(server, ctypes.byref(params), ctypes.byref(jid)), "jz_submit")
    return jid.value


def jz_poll(server, job_id: int):
    """The job's JzResult, or None while it is pending."""
    r = JzResult()
    rc = load().jz_poll(server, int(job_id), ctypes.byref(r))
    if rc == ISING_ERR_PENDING:
        return None
    _check(rc, "jz_poll")
    return r


def jz_wait(server, job_id: int, timeout_s: float = 3600.0) -> JzResult:
    r = JzResult()
    _check(load().jz_wait(server, int(job_id), float(timeout_s), ctypes.byref(r)), "jz_wait")
    return r


def jz_server_work(server, job_id: int, work_out) -> None:
    _check(load().jz_server_work(server, int(job_id), _ptr(work_out)), "jz_server_work")


def jz_server_free(server) -> None:
    load().jz_server_free(server)


def ising_cancel(ctx) -> None:
    """Set the context's cancel flag: run calls refuse new work until reset."""
    _check(load().ising_cancel(ctx), "ising_cancel")


def ising_cancel_reset(ctx) -> None:
    _check(load().ising_cancel_reset(ctx), "ising_cancel_reset")


def jarzynski_run_resumable(ctx, params: JzParams, steps_per_segment: int, work_io, spins_io,
                            k_done: int = 0, max_segments: int = 0):
    """Run the protocol from step k_done in segments, testing the cancel flag
    between them.  Returns (status, k_done): status ISING_OK (finished),
    ISING_ERR_PENDING (max_segments reached) or ISING_ERR_CANCELLED; other
    errors raise IsingError."""
    k = ctypes.c_int(int(k_done))
    rc = load().jarzynski_run_resumable(ctx, ctypes.byref(params), int(steps_per_segment),
                                        int(max_segments), ctypes.byref(k), _ptr(work_io),
                                        _ptr(spins_io))
    if rc not in (ISING_OK, ISING_ERR_PENDING, ISING_ERR_CANCELLED):
        _check(rc, "jarzynski_run_resumable")
    return rc, k.value


def jz_cancel(server, job_id: int) -> None:
    _check(load().jz_cancel(server, int(job_id)), "jz_cancel")


def jz_server_set_log(server, path) -> None:
    """Append one JSON line per finished job to `path` (None: stop logging)."""
    _check(load().jz_server_set_log(server, None if path is None else str(path).encode()),
           "jz_server_set_log")


def jz_result_json(job_id: int, params: JzParams, result: JzResult) -> str:
    buf = ctypes.create_string_buffer(1024)
    n = load().jz_result_json(int(job_id), ctypes.byref(params), ctypes.byref(result), buf, 1024)
    if n < 0:
        _check(n, "jz_result_json")
    return buf.value.decode()


class TuneCache:
    """The persisted autotune cache (see include/isingjz.h); host only."""

    def __init__(self):
        h = ctypes.c_void_p()
        _check(load().jz_tune_cache_create(ctypes.byref(h)), "jz_tune_cache_create")
        self.handle = h.value

    def close(self):
        if self.handle:
            load().jz_tune_cache_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, path):
        _check(load().jz_tune_cache_load(self.handle, str(path).encode()), "jz_tune_cache_load")

    def save(self, path):
        _check(load().jz_tune_cache_save(self.handle, str(path).encode()), "jz_tune_cache_save")

    def put(self, gpu, d, L, L_t, n_replica, n_traj, cta_threads):
        _check(load().jz_tune_cache_put(self.handle, gpu.encode(), int(d), int(L), int(L_t),
                                        int(n_replica), int(n_traj), int(cta_threads)),
               "jz_tune_cache_put")

    def get(self, gpu, d, L, L_t, n_replica, n_traj):
        """The cached CTA size, or None on a miss."""
        t = ctypes.c_int()
        rc = load().jz_tune_cache_get(self.handle, gpu.encode(), int(d), int(L), int(L_t),
                                      int(n_replica), int(n_traj), ctypes.byref(t))
        if rc == ISING_ERR_NOT_FOUND:
            return None
        _check(rc, "jz_tune_cache_get")
        return t.value

    def __len__(self):
        n = ctypes.c_int()
        _check(load().jz_tune_cache_size(self.handle, ctypes.byref(n)), "jz_tune_cache_size")
        return n.value


def ising_autotune_cached(ctx, cache: TuneCache, params: JzParams):
    """(CTA size, hit): the cached choice for the context's GPU, else a fresh
    ising_autotune whose choice is stored in the cache."""
    t, hit = ctypes.c_int(), ctypes.c_int()
    _check(load().ising_autotune_cached(ctx, cache.handle, ctypes.byref(params), ctypes.byref(t),
                                        ctypes.byref(hit)), "ising_autotune_cached")
    return t.value, bool(hit.value)


def ising_bounds_status(clear: bool = False):
    """(failed check sites, one failing index) of the bounds-checked build."""
    a, b = ctypes.c_uint(), ctypes.c_uint()
    _check(load().ising_bounds_status(ctypes.byref(a), ctypes.byref(b), int(bool(clear))),
           "ising_bounds_status")
    return a.value, b.value
