"""ctypes wrapper of the plain CPU oracle (sa_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the smoke check and by
the benchmark's CPU-baseline leg.  Nothing in the product path may import it.
It does not import the CUDA package and shares no code with it.

The oracle follows arXiv:2511.17245 step by step (Sect. 3): it merges terms,
recomputes every energy difference from the definition E(z') - E(z) over the
variable's terms (no cached coefficients), runs the sequential single-variable
sweep with the geometric schedule, and draws moves by Metropolis, heat bath
(explicit inverse CDF) or optimal-transition Metropolis (brute-force argmin).

Parity unpinned: none.  Every exported function has a pin in tests/ (brute
force, closed forms, invariants or published known-answer vectors).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sa_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

RULES = {"metropolis": 0, "heat_bath": 1, "opt_metropolis": 2}
COEF = {"i32": 0, "i64": 1, "f32": 2, "f64": 3}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class FollowStats(C.Structure):
    _fields_ = [("near_threshold", C.c_int64), ("followed", C.c_int64), ("mismatch", C.c_int64),
                ("first_bad_s", C.c_int64), ("first_bad_k", C.c_int64), ("first_bad_r", C.c_int64),
                ("first_bad_oracle", C.c_int64), ("first_bad_trace", C.c_int64)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        P = C.c_void_p
        lib.om_philox4x32_10.argtypes = [P, P, P]
        lib.om_model_create.argtypes = [C.POINTER(C.c_void_p), C.c_int32, P, P, C.c_int64, P, P, P, C.c_int]
        lib.om_model_create.restype = C.c_int
        lib.om_model_destroy.argtypes = [P]
        lib.om_model_n_terms.argtypes = [P]
        lib.om_model_n_terms.restype = C.c_int32
        lib.om_model_is_float.argtypes = [P]
        lib.om_model_flat_len.argtypes = [P]
        lib.om_model_flat_len.restype = C.c_int64
        lib.om_model_terms.argtypes = [P, P, P, P, P]
        lib.om_energy_i.argtypes = [P, P]
        lib.om_energy_i.restype = C.c_int64
        lib.om_energy_f.argtypes = [P, P]
        lib.om_energy_f.restype = C.c_double
        lib.om_delta_i.argtypes = [P, P, C.c_int32, C.c_int64]
        lib.om_delta_i.restype = C.c_int64
        lib.om_delta_f.argtypes = [P, P, C.c_int32, C.c_double]
        lib.om_delta_f.restype = C.c_double
        lib.om_schedule.argtypes = [C.c_int32, C.c_double, C.c_double, P, P, P]
        lib.om_auto_temperatures.argtypes = [P, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        lib.om_run.argtypes = [P, C.c_int, C.c_int32, C.c_uint64, C.c_uint32, C.c_double, C.c_double,
                               C.c_double, C.c_int32, C.c_int32, P, P, C.c_int32, P, P, P, P, P, P,
                               C.POINTER(FollowStats), P, P, P, P, P, P]
        lib.om_run.restype = C.c_int
        lib.om_attempt.argtypes = [P, P, C.c_int32, C.c_int, C.c_float, C.c_float, C.c_uint64,
                                   C.c_uint32, C.c_uint32, C.c_uint32]
        lib.om_attempt.restype = C.c_int64
        lib.om_argmin_change.argtypes = [P, P, C.c_int32]
        lib.om_argmin_change.restype = C.c_int64
        lib.om_transition_row.argtypes = [P, P, C.c_int32, C.c_int, C.c_double, C.c_double, P]
        lib.om_state_count.argtypes = [P, C.c_int64]
        lib.om_state_count.restype = C.c_int64
        lib.om_enumerate.argtypes = [P, C.c_int64, P, P]
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def philox4x32_10(ctr, key):
    """Raw Philox4x32-10 block: ctr = 4 words, key = 2 words -> 4 words."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.om_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def schedule(n_sweeps, t_max, t_min):
    """(T_s as float64, beta_s = fp32(1/T_s), r_s fp32) for s = 0..S-1."""
    lib = _load()
    t = np.zeros(n_sweeps, np.float64)
    b = np.zeros(n_sweeps, np.float32)
    r = np.zeros(n_sweeps, np.float32)
    lib.om_schedule(n_sweeps, t_max, t_min, _ptr(t), _ptr(b), _ptr(r))
    return t, b, r


class Model:
    """Merged QUIO/HUIO model held by the oracle."""

    def __init__(self, inst):
        lib = _load()
        self._lib = lib
        self.n = int(inst["n_vars"])
        self.lower = np.ascontiguousarray(inst["lower"], np.int64)
        self.upper = np.ascontiguousarray(inst["upper"], np.int64)
        offs = np.ascontiguousarray(inst["term_offsets"], np.int64)
        tv = np.ascontiguousarray(inst["term_vars"], np.int32)
        self.coef_type = inst["coef_type"]
        co = np.ascontiguousarray(inst["coeffs"], {"i32": np.int32, "i64": np.int64, "f32": np.float32,
                                                   "f64": np.float64}[self.coef_type])
        h = C.c_void_p()
        rc = lib.om_model_create(C.byref(h), self.n, _ptr(self.lower), _ptr(self.upper),
                                 len(offs) - 1, _ptr(offs), _ptr(tv), _ptr(co), COEF[self.coef_type])
        if rc != 0:
            raise ValueError(f"oracle model rejected (code {rc})")
        self._h = h
        self.is_float = bool(lib.om_model_is_float(h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.om_model_destroy(h)
            self._h = None

    @property
    def n_terms(self):
        return int(self._lib.om_model_n_terms(self._h))

    def terms(self):
        nt = self.n_terms
        offs = np.zeros(nt + 1, np.int64)
        tv = np.zeros(max(1, int(self._lib.om_model_flat_len(self._h))), np.int32)
        ci = np.zeros(max(1, nt), np.int64)
        cf = np.zeros(max(1, nt), np.float64)
        self._lib.om_model_terms(self._h, _ptr(offs), _ptr(tv), _ptr(ci), _ptr(cf))
        return offs, tv[:offs[-1]].copy(), ci[:nt], cf[:nt]

    def energy(self, z):
        z = np.ascontiguousarray(z, np.int32)
        if self.is_float:
            return float(self._lib.om_energy_f(self._h, _ptr(z)))
        return int(self._lib.om_energy_i(self._h, _ptr(z)))

    def energies(self, states):
        states = np.ascontiguousarray(states, np.int32)
        return np.array([self.energy(s) for s in states],
                        dtype=np.float64 if self.is_float else np.int64)

    def delta(self, z, k, v):
        z = np.ascontiguousarray(z, np.int32)
        if self.is_float:
            return float(self._lib.om_delta_f(self._h, _ptr(z), int(k), float(v)))
        return int(self._lib.om_delta_i(self._h, _ptr(z), int(k), int(v)))

    def auto_temperatures(self):
        a, b = C.c_double(), C.c_double()
        self._lib.om_auto_temperatures(self._h, C.byref(a), C.byref(b))
        return a.value, b.value

    def run(self, rule, n_sweeps, seed, t_max, t_min, r_begin=0, r_end=1, instance=0,
            init_states=None, trace=None, trace_replicas=0, margin=1e-6, energy_trace=False,
            record_trace=False, best=False):
        """SA run for replicas [r_begin, r_end); see om_run in sa_oracle.c."""
        R = r_end - r_begin
        out_z = np.zeros((R, self.n), np.int32)
        e_i = np.zeros(R, np.int64)
        e_f = np.zeros(R, np.float64)
        er_i = np.zeros(R, np.int64)
        er_f = np.zeros(R, np.float64)
        ch = np.zeros(R, np.int64)
        st = FollowStats()
        init = None if init_states is None else np.ascontiguousarray(init_states, np.int32)
        tr = None if trace is None else np.ascontiguousarray(trace, np.int32)
        et_i = np.zeros((n_sweeps, R), np.int64) if energy_trace else None
        et_f = np.zeros((n_sweeps, R), np.float64) if energy_trace else None
        tr_out = np.zeros((n_sweeps, R, self.n), np.int32) if record_trace else None
        b_z = np.zeros((R, self.n), np.int32) if best else None
        b_i = np.zeros(R, np.int64) if best else None
        b_f = np.zeros(R, np.float64) if best else None
        rc = self._lib.om_run(self._h, RULES[rule] if isinstance(rule, str) else int(rule), int(n_sweeps),
                              C.c_uint64(seed), C.c_uint32(instance), float(t_max), float(t_min), float(margin),
                              int(r_begin), int(r_end), _ptr(init), _ptr(tr), int(trace_replicas),
                              _ptr(out_z), _ptr(e_i), _ptr(e_f), _ptr(er_i), _ptr(er_f), _ptr(ch),
                              C.byref(st), _ptr(et_i), _ptr(et_f), _ptr(tr_out), _ptr(b_z), _ptr(b_i), _ptr(b_f))
        if rc != 0:
            raise ValueError(f"oracle run rejected (code {rc})")
        res = {"states": out_z, "changes": ch, "follow": st.as_dict()}
        if record_trace:
            res["trace"] = tr_out
        if best:
            res["best_states"] = b_z
            res["best_energy"] = b_f if self.is_float else b_i
        if self.is_float:
            res["energy"] = e_f
            res["energy_recomputed"] = er_f
            if energy_trace:
                res["energy_trace"] = et_f
        else:
            res["energy"] = e_i
            res["energy_recomputed"] = er_i
            if energy_trace:
                res["energy_trace"] = et_i
        return res

    def attempt(self, z, k, rule, beta, ratio, seed, s, r, inst=0):
        z = np.ascontiguousarray(z, np.int32)
        return int(self._lib.om_attempt(self._h, _ptr(z), int(k), RULES[rule] if isinstance(rule, str) else int(rule),
                                        C.c_float(beta), C.c_float(ratio), C.c_uint64(seed),
                                        C.c_uint32(s), C.c_uint32(r), C.c_uint32(inst)))

    def argmin_change(self, z, k):
        z = np.ascontiguousarray(z, np.int32)
        return int(self._lib.om_argmin_change(self._h, _ptr(z), int(k)))

    def transition_row(self, z, k, rule, temp, ratio=0.0):
        z = np.ascontiguousarray(z, np.int32)
        n = int(self.upper[k] - self.lower[k] + 1)
        out = np.zeros(n, np.float64)
        self._lib.om_transition_row(self._h, _ptr(z), int(k), RULES[rule] if isinstance(rule, str) else int(rule),
                                    float(temp), float(ratio), _ptr(out))
        return out

    def enumerate(self, cap=2_000_000):
        cnt = int(self._lib.om_state_count(self._h, cap))
        if cnt == 0:
            raise ValueError("too many states to enumerate")
        e = np.zeros(cnt, np.float64)
        s = np.zeros((cnt, self.n), np.int32)
        self._lib.om_enumerate(self._h, cnt, _ptr(e), _ptr(s))
        return s, e
