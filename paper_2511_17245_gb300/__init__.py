"""GB300 (sm_103a) direct simulated annealing for QUIO/HUIO (arXiv:2511.17245).

The compute path is the CUDA library libsa_gb300.so behind the C ABI of
include/sa.h; `_lib` is its ctypes binding.  `Model` below is a convenience
wrapper that allocates torch tensors for the outputs and forwards to the
C entry points; it performs no arithmetic of the method.
"""
from __future__ import annotations

from . import _lib
from ._lib import (RULES, SAError, make_params, sa_batch_autotune, sa_batch_create, sa_batch_destroy,
                   sa_batch_get_info, sa_batch_result, sa_batch_run, sa_default_temperatures, sa_energy,
                   sa_last_error, sa_measure_peaks, sa_model_create, sa_model_create_quio_dense,
                   sa_model_destroy, sa_model_get_info, sa_run, sa_run_noalloc, sa_run_report, sa_server_cancel,
                   sa_server_create, sa_server_destroy, sa_server_get_stats, sa_server_poll, sa_server_result,
                   sa_server_submit, sa_server_wait, sa_version)

__all__ = ["Model", "RULES", "SAError", "make_params", "sa_batch_autotune", "sa_batch_create", "sa_batch_destroy",
           "sa_batch_get_info", "sa_batch_result", "sa_batch_run", "sa_default_temperatures", "sa_energy",
           "sa_last_error", "sa_measure_peaks", "sa_model_create", "sa_model_create_quio_dense", "sa_model_destroy",
           "sa_model_get_info", "sa_run", "sa_run_noalloc", "sa_run_report", "sa_server_cancel", "sa_server_create",
           "sa_server_destroy", "sa_server_get_stats", "sa_server_poll", "sa_server_result", "sa_server_submit",
           "sa_server_wait", "sa_version"]


class Model:
    """Owns one sa_model handle built from an instance dict (see workloads)."""

    def __init__(self, inst):
        self.n = int(inst["n_vars"])
        if "J" in inst:   # dense QUIO spec
            self.handle = sa_model_create_quio_dense(inst["n_vars"], inst["lower"], inst["upper"], inst["h"],
                                                     inst["J"], inst["coef_type"])
        else:
            self.handle = sa_model_create(inst["n_vars"], inst["lower"], inst["upper"], inst["term_offsets"],
                                          inst["term_vars"], inst["coeffs"], inst["coef_type"])
        self.info = sa_model_get_info(self.handle)
        self.is_float = bool(self.info["is_float"])

    def close(self):
        if getattr(self, "handle", None):
            sa_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def default_temperatures(self):
        return sa_default_temperatures(self.handle)

    def run(self, rule="metropolis", n_sweeps=1000, n_replicas=64, seed=0, device="cuda", stream=None,
            report=False, best=False, **kw):
        """Runs sa_run into freshly allocated torch tensors; returns a dict
        (with best=True also the best states at sweep ends and their energies)."""
        import torch
        edt = torch.float64 if self.is_float else torch.int64
        states = torch.empty((n_replicas, self.n), dtype=torch.int32, device=device)
        energies = torch.empty(n_replicas, dtype=edt, device=device)
        accepts = torch.empty(n_replicas, dtype=torch.int64, device=device)
        if best:
            kw["best_states"] = torch.empty((n_replicas, self.n), dtype=torch.int32, device=device)
            kw["best_energies"] = torch.empty(n_replicas, dtype=edt, device=device)
        rep = sa_run_report() if report else None
        params = make_params(rule=rule, n_sweeps=n_sweeps, n_replicas=n_replicas, seed=seed, report=rep, **kw)
        if stream is None and str(device).startswith("cuda"):
            stream = torch.cuda.current_stream().cuda_stream
        sa_run(self.handle, params, states, energies, accepts, stream)
        out = {"states": states, "energies": energies, "accepts": accepts}
        if best:
            out["best_states"], out["best_energies"] = kw["best_states"], kw["best_energies"]
        if rep is not None:
            out["report"] = {f: getattr(rep, f) for f, _ in rep._fields_}
        return out

    def energy(self, states, stream=None):
        import torch
        n = states.shape[0]
        dev = states.device
        out = torch.empty(n, dtype=torch.float64 if self.is_float else torch.int64, device=dev)
        if stream is None and dev.type == "cuda":
            stream = torch.cuda.current_stream().cuda_stream
        sa_energy(self.handle, states.contiguous(), n, out, stream)
        return out
