"""Batched runs (one persistent, graph-captured launch over many instances)
against per-instance sa_run and the CPU oracle.

Integer instances: every instance's states, energies and change counts equal
those of sa_run with the same parameters (same Philox counters), before and
after autotuning.  Float instances: energies within 1e-5 of an FP64
recomputation, distributions KS-compatible with the oracle.
"""
import concurrent.futures as cf

import numpy as np
import pytest
from scipy import stats

torch = pytest.importorskip("torch")

from oracle import oracle as orc
from paper_2511_17245_gb300 import (Model, make_params, sa_batch_autotune, sa_batch_create, sa_batch_destroy,
                                    sa_batch_get_info, sa_batch_result, sa_batch_run)
from paper_2511_17245_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _batch_results(models, params, autotune=0):
    b = sa_batch_create([m.handle for m in models], params)
    try:
        if autotune:
            sa_batch_autotune(b, autotune)
        sa_batch_run(b)
        torch.cuda.synchronize()
        out = []
        for i, (m, p) in enumerate(zip(models, params)):
            st = np.zeros((p.n_replicas, m.n), np.int32)
            en = np.zeros(p.n_replicas, np.float64 if m.is_float else np.int64)
            ac = np.zeros(p.n_replicas, np.uint64)
            sa_batch_result(b, i, st, en, ac)
            out.append((st, en, ac))
        return out, sa_batch_get_info(b)
    finally:
        sa_batch_destroy(b)


def _int_instances(kind, n_inst, seed):
    rng = np.random.default_rng(seed)
    insts = []
    for i in range(n_inst):
        n = int(rng.integers(5, 120))
        if kind == "quio":
            w = int(rng.integers(1, 300))
            insts.append(wl.quio_sparse_int(seed * 100 + i, n=n, n_edges=min(n * (n - 1) // 2, 3 * n),
                                            lo=-(w // 2), hi=w - w // 2, jmax=4, hmax=30, dmax=3))
        else:
            insts.append(wl.random_small(seed * 100 + i, n=n, max_order=4, lo=-4, hi=5, n_terms=3 * n,
                                         coef_type="i32", cmax=4))
    return insts


@pytest.mark.parametrize("kind", ["quio", "huio"])
@pytest.mark.parametrize("rule", ["metropolis", "heat_bath", "opt_metropolis"])
def test_batch_equals_single_runs_int(kind, rule):
    insts = _int_instances(kind, 24, 7 if kind == "quio" else 8)
    models = [Model(x) for x in insts]
    rng = np.random.default_rng(1)
    params = [make_params(rule, int(rng.integers(5, 60)), int(rng.integers(1, 40)), seed=11, instance_id=i,
                          t_max=float(rng.uniform(20, 200)), t_min=0.5) for i in range(len(models))]
    for tune in (0, 3):
        res, info = _batch_results(models, params, autotune=tune)
        for i, (m, p) in enumerate(zip(models, params)):
            one = m.run(rule, p.n_sweeps, p.n_replicas, seed=11, instance_id=i, t_max=p.t_max, t_min=p.t_min)
            assert np.array_equal(res[i][0], one["states"].cpu().numpy()), (kind, rule, i, tune)
            assert np.array_equal(res[i][1], one["energies"].cpu().numpy()), (kind, rule, i, tune)
            assert np.array_equal(res[i][2].astype(np.int64), one["accepts"].cpu().numpy()), (kind, rule, i, tune)
        assert info["n_units"] == sum(p.n_replicas for p in params)


def test_dense_model_equals_term_list():
    spec = {"index": 0, "n": 150, "width": 37, "dense": True, "deg": 0, "seed": 5}
    dense = wl.batch_instance(spec)
    terms = wl.batch_instance(spec, as_terms=True)
    a, b = Model(dense), Model(terms)
    assert a.info["n_terms"] == b.info["n_terms"] and a.info["n_levels"] == b.info["n_levels"] == 150
    st = torch.from_numpy(wl.initial_states(2, terms, 20)).cuda()
    assert torch.equal(a.energy(st), b.energy(st))
    ra = a.run("heat_bath", 30, 8, seed=4, t_max=50.0, t_min=0.1)
    rb = b.run("heat_bath", 30, 8, seed=4, t_max=50.0, t_min=0.1)
    np.testing.assert_allclose(ra["energies"].cpu().numpy(), rb["energies"].cpu().numpy(), rtol=1e-5)


def test_batch_float_instances():
    specs = wl.batch_specs(9, n_instances=40, n_min=20, n_max=300, w_min=2, w_max=64)
    insts = [wl.batch_instance(s) for s in specs]
    models = [Model(x) for x in insts]
    params = []
    for i, m in enumerate(models):
        tmax, tmin = m.default_temperatures()
        params.append(make_params("metropolis", 200, 32, seed=0, instance_id=i, t_max=tmax, t_min=tmin))
    res, info = _batch_results(models, params, autotune=5)
    for i, m in enumerate(models):
        st = torch.from_numpy(res[i][0]).cuda()
        np.testing.assert_allclose(res[i][1], m.energy(st).cpu().numpy(), rtol=1e-5, atol=1e-6)
    # two sparse instances against the oracle (32 device vs 32 oracle replicas)
    picked = [i for i, s in enumerate(specs) if not s["dense"]][:2]
    for i in picked:
        om = orc.Model(wl.batch_instance(specs[i]))
        p = params[i]
        with cf.ThreadPoolExecutor(max_workers=8) as ex:
            o = list(ex.map(lambda r: om.run("metropolis", 200, 0, p.t_max, p.t_min, r_begin=r, r_end=r + 1,
                                             instance=i), range(32)))
        eo = np.array([x["energy"][0] for x in o])
        assert stats.ks_2samp(res[i][1], eo).pvalue > 0.01, i


@pytest.mark.parametrize("rule", ["metropolis", "heat_bath", "opt_metropolis"])
def test_batch_speculative_equals_level_order(rule):
    """A batch mixing complete, nearly complete, path-like and sparse integer
    instances gives, with speculative windows, the states, energies and change
    counts of the level-by-level order bit for bit, before and after autotuning."""
    from paper_2511_17245_gb300 import _lib
    insts = []
    for i in range(4):
        insts.append(wl.quio_complete(20 + i, n=40 + 60 * i, lo=-20, hi=20))
        insts.append(wl.quio_dense_small(30 + i, n=30 + 40 * i, lo=-8, hi=7))
        insts.append(wl.quio_chain(40 + i, n=100 + 50 * i, lo=-30, hi=30, n_long=10 * i))
        insts.append(wl.quio_sparse_int(50 + i, n=150, n_edges=600, lo=-5, hi=5))
    models = [Model(x) for x in insts]
    runs = []
    for flags in (_lib.SA_FLAG_NO_SPECULATION, 0):
        params = []
        for i, m in enumerate(models):
            tmax, tmin = m.default_temperatures()
            params.append(make_params(rule, 60, 16, seed=1, instance_id=i, t_max=tmax, t_min=tmin, flags=flags))
        runs.append(_batch_results(models, params)[0])
        if flags == 0:
            runs.append(_batch_results(models, params, autotune=3)[0])
    for got in runs[1:]:
        for i in range(len(models)):
            for j in range(3):
                np.testing.assert_array_equal(runs[0][i][j], got[i][j], err_msg=f"instance {i} output {j}")


def test_batch_full_size_sampled():
    """4,096 instances (N log-uniform in [50, 2000], range width log-uniform in
    [2, 1024], half dense / half sparse with degree 8..64), 32 replicas, 1000
    sweeps, Metropolis, temperatures of Sect. 3.4 per instance: one batched
    launch.  Every instance's energies are within 1e-5 of an FP64
    recomputation of its states; two small sparse instances are KS-compatible
    with the oracle."""
    specs = wl.batch_specs(3)
    models, params = [], []
    for i, s in enumerate(specs):
        m = Model(wl.batch_instance(s))
        tmax, tmin = m.default_temperatures()
        models.append(m)
        params.append(make_params("metropolis", 1000, 32, seed=0, instance_id=i, t_max=tmax, t_min=tmin))
    b = sa_batch_create([m.handle for m in models], params)
    try:
        sa_batch_run(b)
        torch.cuda.synchronize()
        info = sa_batch_get_info(b)
        assert info["n_units"] == 4096 * 32
        rng = np.random.default_rng(0)
        check = rng.choice(4096, size=256, replace=False)
        small_sparse = [i for i, s in enumerate(specs) if not s["dense"] and s["n"] < 120][:2]
        for i in list(check) + small_sparse:
            m = models[i]
            st = torch.zeros((32, m.n), dtype=torch.int32, device="cuda")
            en = torch.zeros(32, dtype=torch.float64, device="cuda")
            sa_batch_result(b, int(i), st, en, None, torch.cuda.current_stream().cuda_stream)
            np.testing.assert_allclose(en.cpu().numpy(), m.energy(st).cpu().numpy(), rtol=1e-5, atol=1e-6)
        for i in small_sparse:
            om = orc.Model(wl.batch_instance(specs[i]))
            p = params[i]
            en = np.zeros(32, np.float64)
            sa_batch_result(b, i, None, en, None)
            with cf.ThreadPoolExecutor(max_workers=8) as ex:
                o = list(ex.map(lambda r: om.run("metropolis", 1000, 0, p.t_max, p.t_min, r_begin=r, r_end=r + 1,
                                                 instance=i), range(32)))
            eo = np.array([x["energy"][0] for x in o])
            assert stats.ks_2samp(en, eo).pvalue > 0.01, i
    finally:
        sa_batch_destroy(b)
