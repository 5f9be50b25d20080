"""Thin ctypes binding of the C ABI in include/sa.h (libsa_gb300.so).

Argument marshalling only: every step of the SA sweep runs in the CUDA
library.  Functions keep the C names.  Buffers may be torch tensors (device or
host) or numpy arrays (host); their raw pointers are passed through.  There is
no CPU fallback: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsa_gb300.so")
_lock = threading.Lock()
_lib = None

SA_OK, SA_ERR_INVALID, SA_ERR_OVERFLOW, SA_ERR_UNSUPPORTED, SA_ERR_OOM, SA_ERR_CUDA, SA_ERR_TIMEOUT, SA_ERR_BUSY = range(8)
STATUS_NAMES = ["SA_OK", "SA_ERR_INVALID", "SA_ERR_OVERFLOW", "SA_ERR_UNSUPPORTED", "SA_ERR_OOM",
                "SA_ERR_CUDA", "SA_ERR_TIMEOUT", "SA_ERR_BUSY"]
COEF = {"i32": 0, "i64": 1, "f32": 2, "f64": 3}
RULES = {"metropolis": 0, "heat_bath": 1, "opt_metropolis": 2}
SA_FLAG_STATE_IN_GLOBAL = 0x1
SA_FLAG_NO_TIME_SLICING = 0x2
SA_FLAG_NO_SPECULATION = 0x4


class SAError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class sa_model_info(C.Structure):
    _fields_ = [("n_vars", C.c_int32), ("is_float", C.c_int32), ("is_quadratic", C.c_int32),
                ("max_exponent", C.c_int32), ("max_order", C.c_int32), ("all_multilinear", C.c_int32),
                ("n_terms", C.c_int64), ("n_links", C.c_int64), ("n_levels", C.c_int32),
                ("max_width", C.c_int32), ("device_bytes", C.c_int64)]


class sa_run_report(C.Structure):
    _fields_ = [("max_refresh_drift", C.c_double), ("replicas_per_block", C.c_int32),
                ("threads_per_replica", C.c_int32), ("state_in_global", C.c_int32), ("shared_bytes", C.c_int32),
                ("blocks", C.c_int32), ("n_levels", C.c_int32), ("kernel_ms", C.c_float), ("time_sliced", C.c_int32)]


class sa_batch_info(C.Structure):
    _fields_ = [("n_instances", C.c_int32), ("n_units", C.c_int32), ("replicas_per_block", C.c_int32),
                ("threads_per_replica", C.c_int32), ("blocks", C.c_int32), ("state_in_global", C.c_int32),
                ("attempts", C.c_int64), ("device_bytes", C.c_int64), ("autotune_ms", C.c_float),
                ("_reserved", C.c_int32)]


class sa_server_config(C.Structure):
    _fields_ = [("budget_bytes", C.c_uint64), ("max_running", C.c_int32), ("threads_per_replica", C.c_int32)]


class sa_server_stats(C.Structure):
    _fields_ = [("completed", C.c_int64), ("failed", C.c_int64), ("cancelled", C.c_int64), ("queued", C.c_int64),
                ("running", C.c_int64), ("device_bytes_in_use", C.c_int64), ("device_bytes_peak", C.c_int64),
                ("attempts", C.c_int64), ("p50_latency_ms", C.c_double), ("p99_latency_ms", C.c_double),
                ("attempts_per_s", C.c_double), ("units_done", C.c_int64), ("kernel_launches", C.c_int64)]


class sa_peaks(C.Structure):
    _fields_ = [("exp2_per_s", C.c_double), ("fma_per_s", C.c_double), ("l2_gbs", C.c_double),
                ("smem_gbs", C.c_double), ("smem_atomic_per_s", C.c_double), ("sms", C.c_int32),
                ("l2_buffer_bytes", C.c_int32), ("exp2_ms", C.c_float), ("fma_ms", C.c_float),
                ("l2_ms", C.c_float), ("smem_ms", C.c_float), ("smem_atomic_ms", C.c_float)]


class sa_run_params(C.Structure):
    _fields_ = [("rule", C.c_int32), ("n_sweeps", C.c_int32), ("n_replicas", C.c_int32),
                ("refresh_interval", C.c_int32), ("seed", C.c_uint64), ("t_max", C.c_double),
                ("t_min", C.c_double), ("temperatures", C.c_void_p), ("init_states", C.c_void_p),
                ("instance_id", C.c_uint32), ("replicas_per_block", C.c_int32),
                ("threads_per_replica", C.c_int32), ("flags", C.c_int32), ("trace", C.c_void_p),
                ("trace_replicas", C.c_int32), ("_pad0", C.c_int32), ("energy_trace", C.c_void_p),
                ("report", C.POINTER(sa_run_report)), ("best_states", C.c_void_p), ("best_energies", C.c_void_p)]


# Every symbol include/*.h declares (checked by the tests).
EXPORTS = ["sa_model_create", "sa_model_destroy", "sa_model_get_info", "sa_default_temperatures",
           "sa_run", "sa_energy", "sa_last_error", "sa_version", "sa_run_noalloc", "sa_model_create_quio_dense",
           "sa_batch_create", "sa_batch_autotune", "sa_batch_run", "sa_batch_result", "sa_batch_get_info",
           "sa_batch_destroy", "sa_server_create", "sa_server_submit", "sa_server_poll", "sa_server_wait",
           "sa_server_cancel", "sa_server_result", "sa_server_get_stats", "sa_server_destroy",
           "sa_measure_peaks"]
SA_REQ_QUEUED, SA_REQ_RUNNING, SA_REQ_DONE, SA_REQ_FAILED, SA_REQ_CANCELLED = range(5)
# size of the fixed device scratch array behind sa_run_noalloc (SA_NOALLOC_SCRATCH_BYTES)
NOALLOC_SCRATCH_BYTES = 4 << 20


def load():
    """Loads libsa_gb300.so (built by paper_2511_17245_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = C.CDLL(LIB_PATH)
        P = C.c_void_p
        lib.sa_model_create.argtypes = [C.POINTER(C.c_void_p), C.c_int32, P, P, C.c_int64, P, P, P, C.c_int]
        lib.sa_model_create.restype = C.c_int
        lib.sa_model_destroy.argtypes = [P]
        lib.sa_model_destroy.restype = None
        lib.sa_model_get_info.argtypes = [P, C.POINTER(sa_model_info)]
        lib.sa_model_get_info.restype = C.c_int
        lib.sa_default_temperatures.argtypes = [P, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        lib.sa_default_temperatures.restype = C.c_int
        lib.sa_run.argtypes = [P, C.POINTER(sa_run_params), P, P, P, P]
        lib.sa_run.restype = C.c_int
        lib.sa_run_noalloc.argtypes = [P, C.POINTER(sa_run_params), P, P, P, P]
        lib.sa_run_noalloc.restype = C.c_int
        lib.sa_model_create_quio_dense.argtypes = [C.POINTER(C.c_void_p), C.c_int32, P, P, P, P, C.c_int]
        lib.sa_model_create_quio_dense.restype = C.c_int
        lib.sa_batch_create.argtypes = [C.POINTER(C.c_void_p), P, C.c_int32, P]
        lib.sa_batch_create.restype = C.c_int
        lib.sa_batch_autotune.argtypes = [P, C.c_int32, P]
        lib.sa_batch_autotune.restype = C.c_int
        lib.sa_batch_run.argtypes = [P, P]
        lib.sa_batch_run.restype = C.c_int
        lib.sa_batch_result.argtypes = [P, C.c_int32, P, P, P, P]
        lib.sa_batch_result.restype = C.c_int
        lib.sa_batch_get_info.argtypes = [P, C.POINTER(sa_batch_info)]
        lib.sa_batch_get_info.restype = C.c_int
        lib.sa_batch_destroy.argtypes = [P]
        lib.sa_batch_destroy.restype = None
        lib.sa_server_create.argtypes = [C.POINTER(C.c_void_p), C.POINTER(sa_server_config)]
        lib.sa_server_create.restype = C.c_int
        lib.sa_server_submit.argtypes = [P, P, C.POINTER(sa_run_params), C.POINTER(C.c_uint64)]
        lib.sa_server_submit.restype = C.c_int
        lib.sa_server_poll.argtypes = [P, C.c_uint64, C.POINTER(C.c_int32)]
        lib.sa_server_poll.restype = C.c_int
        lib.sa_server_wait.argtypes = [P, C.c_uint64, C.c_int64]
        lib.sa_server_wait.restype = C.c_int
        lib.sa_server_cancel.argtypes = [P, C.c_uint64]
        lib.sa_server_cancel.restype = C.c_int
        lib.sa_server_result.argtypes = [P, C.c_uint64, P, P, P, C.POINTER(C.c_double)]
        lib.sa_server_result.restype = C.c_int
        lib.sa_server_get_stats.argtypes = [P, C.POINTER(sa_server_stats)]
        lib.sa_server_get_stats.restype = C.c_int
        lib.sa_server_destroy.argtypes = [P]
        lib.sa_server_destroy.restype = None
        lib.sa_measure_peaks.argtypes = [C.POINTER(sa_peaks), P]
        lib.sa_measure_peaks.restype = C.c_int
        lib.sa_energy.argtypes = [P, P, C.c_int64, P, P]
        lib.sa_energy.restype = C.c_int
        lib.sa_last_error.argtypes = []
        lib.sa_last_error.restype = C.c_char_p
        lib.sa_version.argtypes = []
        lib.sa_version.restype = C.c_char_p
        _lib = lib
        return lib


def ptr(x):
    """Raw address of a torch tensor / numpy array / int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _check(rc):
    if rc != SA_OK:
        raise SAError(rc, sa_last_error())


def sa_last_error() -> str:
    return load().sa_last_error().decode()


def sa_version() -> str:
    return load().sa_version().decode()


def sa_model_create(n_vars, lower, upper, term_offsets, term_vars, coeffs, coef_type):
    """Returns an opaque model handle (int).  Host arrays in."""
    lib = load()
    lower = np.ascontiguousarray(lower, np.int64)
    upper = np.ascontiguousarray(upper, np.int64)
    term_offsets = np.ascontiguousarray(term_offsets, np.int64)
    term_vars = np.ascontiguousarray(term_vars, np.int32)
    ct = COEF[coef_type] if isinstance(coef_type, str) else int(coef_type)
    dt = {0: np.int32, 1: np.int64, 2: np.float32, 3: np.float64}[ct]
    coeffs = np.ascontiguousarray(coeffs, dt)
    h = C.c_void_p()
    _check(lib.sa_model_create(C.byref(h), int(n_vars), ptr(lower), ptr(upper), len(term_offsets) - 1,
                               ptr(term_offsets), ptr(term_vars), ptr(coeffs), ct))
    return h.value


def sa_model_destroy(h):
    if h:
        load().sa_model_destroy(h)


def sa_model_get_info(h) -> dict:
    info = sa_model_info()
    _check(load().sa_model_get_info(h, C.byref(info)))
    return {f: getattr(info, f) for f, _ in info._fields_}


def sa_default_temperatures(h):
    a, b = C.c_double(), C.c_double()
    _check(load().sa_default_temperatures(h, C.byref(a), C.byref(b)))
    return a.value, b.value


def make_params(rule="metropolis", n_sweeps=1000, n_replicas=64, seed=0, t_max=0.0, t_min=0.0,
                temperatures=None, init_states=None, refresh_interval=0, instance_id=0,
                replicas_per_block=0, threads_per_replica=0, flags=0, trace=None, trace_replicas=0,
                energy_trace=None, report=None, best_states=None, best_energies=None):
    p = sa_run_params()
    p.rule = RULES[rule] if isinstance(rule, str) else int(rule)
    p.n_sweeps = int(n_sweeps)
    p.n_replicas = int(n_replicas)
    p.refresh_interval = int(refresh_interval)
    p.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    p.t_max = float(t_max)
    p.t_min = float(t_min)
    p.temperatures = ptr(temperatures)
    p.init_states = ptr(init_states)
    p.instance_id = int(instance_id)
    p.replicas_per_block = int(replicas_per_block)
    p.threads_per_replica = int(threads_per_replica)
    p.flags = int(flags)
    p.trace = ptr(trace)
    p.trace_replicas = int(trace_replicas)
    p.energy_trace = ptr(energy_trace)
    p.report = C.pointer(report) if report is not None else None
    p.best_states = ptr(best_states)
    p.best_energies = ptr(best_energies)
    return p


def sa_run(h, params: sa_run_params, out_states, out_energies, out_accepts=None, stream=None):
    _check(load().sa_run(h, C.byref(params), ptr(out_states), ptr(out_energies), ptr(out_accepts), stream))


def sa_run_noalloc(h, params: sa_run_params, out_states, out_energies, out_accepts=None, stream=None):
    """sa_run for callers that cannot allocate: device buffers only; the run's
    scratch is the library's fixed device array (see include/sa.h)."""
    _check(load().sa_run_noalloc(h, C.byref(params), ptr(out_states), ptr(out_energies), ptr(out_accepts), stream))


def sa_measure_peaks(stream=None) -> dict:
    """Measured SFU exp2, FMA, L2-copy and shared-memory ceilings of the current
    device (include/sa_peaks.h)."""
    pk = sa_peaks()
    _check(load().sa_measure_peaks(C.byref(pk), stream))
    return {f: getattr(pk, f) for f, _ in pk._fields_}


def sa_energy(h, states, n_states, energies, stream=None):
    _check(load().sa_energy(h, ptr(states), int(n_states), ptr(energies), stream))


def sa_model_create_quio_dense(n_vars, lower, upper, h, J, coef_type):
    """Dense QUIO model from h[n] and the row-major n x n matrix J (upper triangle read)."""
    lib = load()
    ct = COEF[coef_type] if isinstance(coef_type, str) else int(coef_type)
    dt = {0: np.int32, 1: np.int64, 2: np.float32, 3: np.float64}[ct]
    lower = np.ascontiguousarray(lower, np.int64)
    upper = np.ascontiguousarray(upper, np.int64)
    h = np.ascontiguousarray(h, dt)
    J = np.ascontiguousarray(J, dt)
    out = C.c_void_p()
    _check(lib.sa_model_create_quio_dense(C.byref(out), int(n_vars), ptr(lower), ptr(upper), ptr(h), ptr(J), ct))
    return out.value


def sa_batch_create(handles, params_list):
    """handles: model handles; params_list: sa_run_params, one per model."""
    lib = load()
    n = len(handles)
    harr = (C.c_void_p * n)(*handles)
    parr = (sa_run_params * n)(*params_list)
    out = C.c_void_p()
    _check(lib.sa_batch_create(C.byref(out), C.cast(harr, C.c_void_p), n, C.cast(parr, C.c_void_p)))
    return out.value


def sa_batch_autotune(b, trial_sweeps, stream=None):
    _check(load().sa_batch_autotune(b, int(trial_sweeps), stream))


def sa_batch_run(b, stream=None):
    _check(load().sa_batch_run(b, stream))


def sa_batch_result(b, i, states=None, energies=None, accepts=None, stream=None):
    _check(load().sa_batch_result(b, int(i), ptr(states), ptr(energies), ptr(accepts), stream))


def sa_batch_get_info(b) -> dict:
    info = sa_batch_info()
    _check(load().sa_batch_get_info(b, C.byref(info)))
    return {f: getattr(info, f) for f, _ in info._fields_}


def sa_batch_destroy(b):
    if b:
        load().sa_batch_destroy(b)


def sa_server_create(budget_bytes, max_running=1024, threads_per_replica=0):
    cfg = sa_server_config(int(budget_bytes), int(max_running), int(threads_per_replica))
    out = C.c_void_p()
    _check(load().sa_server_create(C.byref(out), C.byref(cfg)))
    return out.value


def sa_server_submit(srv, model_handle, params: sa_run_params):
    t = C.c_uint64()
    _check(load().sa_server_submit(srv, model_handle, C.byref(params), C.byref(t)))
    return t.value


def sa_server_poll(srv, ticket):
    st = C.c_int32()
    _check(load().sa_server_poll(srv, C.c_uint64(ticket), C.byref(st)))
    return st.value


def sa_server_wait(srv, ticket, timeout_us):
    _check(load().sa_server_wait(srv, C.c_uint64(ticket), int(timeout_us)))


def sa_server_cancel(srv, ticket):
    _check(load().sa_server_cancel(srv, C.c_uint64(ticket)))


def sa_server_result(srv, ticket, states=None, energies=None, accepts=None):
    lat = C.c_double()
    _check(load().sa_server_result(srv, C.c_uint64(ticket), ptr(states), ptr(energies), ptr(accepts), C.byref(lat)))
    return lat.value


def sa_server_get_stats(srv) -> dict:
    st = sa_server_stats()
    _check(load().sa_server_get_stats(srv, C.byref(st)))
    return {f: getattr(st, f) for f, _ in st._fields_}


def sa_server_destroy(srv):
    if srv:
        load().sa_server_destroy(srv)
