"""sa_run_noalloc: the SA run for callers that cannot allocate device memory.

Some callers may not call cudaMalloc or cudaFree: code inside a host framework
that owns all device memory through its own arena, or a latency-critical path
where an allocation (which can synchronise the device) is not acceptable.
sa_run_noalloc takes device buffers for every input and output and keeps its
own scratch in a fixed device array of the library.  These tests call it
through the C ABI and check that it returns what sa_run returns, on two calls
in a row (the shared array keeps the previous call's contents), and that it
rejects sizes beyond its fixed scratch with a clear error.

This file is named to be collected last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2511_17245_gb300 import Model, SAError, make_params, sa_energy, sa_run_noalloc
from paper_2511_17245_gb300 import _lib
from paper_2511_17245_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _noalloc(model, rule, S, R, seed, **kw):
    states = torch.empty((R, model.n), dtype=torch.int32, device="cuda")
    energies = torch.empty(R, dtype=torch.float64 if model.is_float else torch.int64, device="cuda")
    accepts = torch.empty(R, dtype=torch.int64, device="cuda")
    p = make_params(rule, S, R, seed=seed, **kw)
    sa_run_noalloc(model.handle, p, states, energies, accepts, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return {"states": states, "energies": energies, "accepts": accepts}


def _same(a, b):
    return all(torch.equal(a[k], b[k]) for k in ("states", "energies", "accepts"))


@pytest.mark.parametrize("rule", ["metropolis", "heat_bath", "opt_metropolis"])
def test_noalloc_equals_sa_run_twice(rule):
    """Integer models: bit-identical to sa_run on two calls in a row, with a call
    on another model (different scratch use) in between."""
    a = Model(wl.huio_zipf(5, n=400, n_quad=800, n_cubic=1200, n_quartic=300, lo=-12, hi=12))
    b = Model(wl.quio_dense_small(2))
    kw = dict(t_max=200.0, t_min=0.5)
    ref_a = a.run(rule, 60, 40, seed=7, **kw)
    ref_b = b.run(rule, 90, 20, seed=8, **kw)
    first = _noalloc(a, rule, 60, 40, 7, **kw)
    other = _noalloc(b, rule, 90, 20, 8, **kw)
    second = _noalloc(a, rule, 60, 40, 7, **kw)
    assert _same(first, ref_a)
    assert _same(second, ref_a)
    assert _same(other, ref_b)


def test_noalloc_state_in_scratch_slab():
    """Replica state kept in the fixed scratch (global placement) instead of
    shared memory: same results as sa_run on two calls, with a run of another
    model in between (other replica count, other state size and layout) that
    leaves its own data in the array, so that a byte read before it is written
    would show."""
    m = Model(wl.huio_zipf(6, n=300, n_quad=600, n_cubic=900, n_quartic=200, lo=-9, hi=9))
    other = Model(wl.quio_sparse_int(9, n=517, n_edges=2100, lo=-70, hi=900, jmax=5, hmax=40, dmax=3))
    glob = _lib.SA_FLAG_STATE_IN_GLOBAL
    kw = dict(t_max=300.0, t_min=1.0, flags=glob)
    ref = m.run("metropolis", 40, 12, seed=3, **kw)
    ref_other = other.run("heat_bath", 25, 29, seed=5, t_max=80.0, t_min=0.5, flags=glob)
    first = _noalloc(m, "metropolis", 40, 12, 3, **kw)
    mid = _noalloc(other, "heat_bath", 25, 29, 5, t_max=80.0, t_min=0.5, flags=glob)
    second = _noalloc(m, "metropolis", 40, 12, 3, **kw)
    assert _same(first, ref)
    assert _same(mid, ref_other)
    assert _same(second, ref)


def test_noalloc_float_model_within_tolerance():
    """Float model: energies within 1e-5 of the FP64 recomputation, and the same
    final-energy distribution as sa_run (KS p > 0.01), twice."""
    from scipy import stats
    m = Model(wl.quio_sparse_wide(12, n=800, n_edges=4000, lo=0, hi=31))
    tmax, tmin = m.default_temperatures()
    ref = m.run("heat_bath", 60, 256, seed=4, t_max=tmax, t_min=tmin).get("energies").cpu().numpy()
    for _ in range(2):
        out = _noalloc(m, "heat_bath", 60, 256, 4, t_max=tmax, t_min=tmin)
        e = out["energies"].cpu().numpy()
        np.testing.assert_allclose(e, m.energy(out["states"]).cpu().numpy(), rtol=1e-5)
        assert stats.ks_2samp(e, ref).pvalue > 0.01


def test_noalloc_rejects_beyond_limits():
    m = Model(wl.quio_dense_small(0))
    too_many = _lib.NOALLOC_SCRATCH_BYTES // 8 + 1
    with pytest.raises(SAError) as e:
        _noalloc(m, "metropolis", too_many, 2, 0, t_max=1.0, t_min=0.5)
    assert e.value.status == _lib.SA_ERR_UNSUPPORTED and "scratch" in str(e.value)
    big = Model(wl.quio_sparse_int(3, n=2000, n_edges=4000, lo=0, hi=7))
    with pytest.raises(SAError) as e:
        _noalloc(big, "metropolis", 2, 300, 0, t_max=1.0, t_min=0.5, flags=_lib.SA_FLAG_STATE_IN_GLOBAL)
    assert e.value.status == _lib.SA_ERR_UNSUPPORTED
    host = np.zeros((2, m.n), np.int32)
    with pytest.raises(SAError) as e:
        sa_run_noalloc(m.handle, make_params("metropolis", 2, 2, t_max=1.0, t_min=0.5), host,
                       np.zeros(2, np.int64), None, None)
    assert e.value.status == _lib.SA_ERR_INVALID
