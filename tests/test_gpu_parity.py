"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer models: the device writes the value of z_k after every attempt of the
traced replicas; the oracle replays the same Philox streams and follows the
device only where a decision lies within the stated margin of its threshold
(1e-6 relative, Metropolis |U - p| <= 1e-6 p, heat bath |U C - C_v| <= 1e-6 C).
Any other difference fails.  Final states, energies (int64) and change counts
must then agree exactly.  Float models: final energies within 1e-5 relative of
an FP64 recomputation, and final-energy distributions over replicas equal to
the oracle's by a two-sample KS test at p > 0.01.
"""
import concurrent.futures as cf
import os

import numpy as np
import pytest
from scipy import stats

torch = pytest.importorskip("torch")

from oracle import oracle as orc
from paper_2511_17245_gb300 import Model, make_params, sa_run, sa_run_report, RULES
from paper_2511_17245_gb300 import _lib
from paper_2511_17245_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
MARGIN = 1e-6
ALL_RULES = ["metropolis", "heat_bath", "opt_metropolis"]


def _device_run(model, rule, S, R, seed, tmax, tmin, trace_R=0, **kw):
    n = model.n
    trace = torch.zeros((S, trace_R, n), dtype=torch.int32, device="cuda") if trace_R else None
    out = model.run(rule=rule, n_sweeps=S, n_replicas=R, seed=seed, t_max=tmax, t_min=tmin,
                    trace=trace, trace_replicas=trace_R, **kw)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items() if hasattr(v, "cpu")}
    if trace is not None:
        res["trace"] = trace.cpu().numpy()
    return res


WORKERS = max(4, os.cpu_count() or 4)


def _oracle_follow(om, rule, S, seed, tmax, tmin, replicas, trace, trace_R, workers=WORKERS, best=False):
    def one(r):
        return om.run(rule, S, seed, tmax, tmin, r_begin=r, r_end=r + 1, trace=trace, trace_replicas=trace_R,
                      margin=MARGIN, best=best)
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        return list(ex.map(one, replicas))


def _check_int_parity(inst, rule, S, R, seed, trace_R, tmax=None, tmin=None, label="", **kw):
    model = Model(inst)
    om = orc.Model(inst)
    if tmax is None:
        tmax, tmin = om.auto_temperatures()
        dt = model.default_temperatures()
        assert dt[0] == pytest.approx(tmax, rel=1e-12) and dt[1] == pytest.approx(tmin, rel=1e-12)
    dev = _device_run(model, rule, S, R, seed, tmax, tmin, trace_R=trace_R, **kw)
    # property at any size: device energies equal the oracle energy of the device states
    for r in range(R):
        assert om.energy(dev["states"][r]) == dev["energies"][r], (label, r)
    assert np.all(dev["states"] >= inst["lower"]) and np.all(dev["states"] <= inst["upper"])
    res = _oracle_follow(om, rule, S, seed, tmax, tmin, list(range(trace_R)), dev["trace"], trace_R)
    near = sum(x["follow"]["near_threshold"] for x in res)
    followed = sum(x["follow"]["followed"] for x in res)
    for r, x in enumerate(res):
        f = x["follow"]
        assert f["mismatch"] == 0, (label, rule, r, f)
        assert np.array_equal(x["states"][0], dev["states"][r]), (label, rule, r)
        assert x["energy"][0] == dev["energies"][r]
        assert x["changes"][0] == dev["accepts"][r]
    print(f"[parity] {label} {rule}: replicas={trace_R} near-threshold={near} followed={followed}")
    return dev


# ------------------------------------------------------------------ integer QUIO
@pytest.mark.parametrize("rule", ALL_RULES)
def test_quio_dense_small_full_size(rule):
    """N=32, z in [-8,7], dense int J, 64 replicas, 1000 sweeps, T 100 -> 0.1:
    every replica traced and replayed."""
    inst = wl.quio_dense_small(0)
    _check_int_parity(inst, rule, 1000, 64, 0, 64, tmax=100.0, tmin=0.1, label="dense-32")


@pytest.mark.parametrize("rule", ALL_RULES)
@pytest.mark.parametrize("lo,hi", [(0, 255), (-300, 300), (-40000, 40000)])
def test_quio_sparse_int_widths(rule, lo, hi):
    """Sparse integer QUIO with 1-, 2- and 4-byte state offsets; ragged N."""
    S = 40 if rule != "heat_bath" or hi - lo < 1000 else 3
    inst = wl.quio_sparse_int(7, n=333, n_edges=1500, lo=lo, hi=hi, jmax=3, hmax=50, dmax=2)
    _check_int_parity(inst, rule, S, 37, 5, 4, label=f"sparse[{lo},{hi}]")


# ------------------------------------------------------------------ integer HUIO
@pytest.mark.parametrize("rule", ALL_RULES)
def test_huio_random_interaction_powers(rule):
    """RI-style terms with repeated indices (exponents up to 4), integer J."""
    inst = wl.random_interaction(40, 4, 6, n_terms=300, seed=3, integer=True, int_scale=20)
    _check_int_parity(inst, rule, 60, 24, 11, 8, label="RI p=4 u=6")


@pytest.mark.parametrize("rule", ALL_RULES)
def test_huio_random_interaction_u100(rule):
    """E^RI_{4,100} (Sect. 4) with integer J: exponents up to 4 over 201 values
    per variable.  Every attempt is replayed against the oracle, whose OTM
    proposal is the brute-force argmin over all 200 changes, so the degree-3/4
    bracketing of the kernel's argmin is checked wherever a proposal is taken."""
    inst = wl.random_interaction(60, 4, 100, n_terms=1000, seed=5, integer=True, int_scale=50)
    S = {"metropolis": 300, "heat_bath": 40, "opt_metropolis": 150}[rule]
    _check_int_parity(inst, rule, S, 16, 5, 6, label="RI p=4 u=100")


@pytest.mark.parametrize("rule", ALL_RULES)
def test_huio_quartic_wells_wide(rule):
    """Tilted double wells a z^4 - 2 a w^2 z^2 + c z^3 + h z over [-1000, 1000],
    ring-coupled: quartic energy differences with two interior minima (OTM
    argmin against brute force over 2000 changes) and heat-bath draws over 2001
    values, replayed attempt by attempt."""
    inst = wl.quartic_wells(3)
    S = {"metropolis": 400, "heat_bath": 60, "opt_metropolis": 300}[rule]
    _check_int_parity(inst, rule, S, 24, 7, 8, label="quartic wells +-1000")


@pytest.mark.parametrize("rule", ALL_RULES)
def test_huio_multilinear_closed_form(rule):
    """Multilinear model (heat bath via the O(1) inverse transform)."""
    inst = wl.multilinear(50, 3, 7, integer=True)
    _check_int_parity(inst, rule, 80, 16, 2, 8, label="ML p=3 u=7")


@pytest.mark.parametrize("rule", ALL_RULES)
def test_huio_zipf_full_size_sampled(rule):
    """N=2000, z in [-50,50], 8k/20k/5k quadratic/cubic/quartic terms with
    Zipf-skewed degrees, 256 replicas at full size; two replicas traced and
    replayed (fewer sweeps for the oracle-heavy heat bath), every replica's
    energy checked against the oracle's energy of its final state."""
    inst = wl.huio_zipf(2)
    S = {"metropolis": 300, "heat_bath": 40, "opt_metropolis": 300}[rule]
    _check_int_parity(inst, rule, S, 256, 0, 2, label="huio-zipf-2000")


SPEC_CASES = {
    # every level one variable, rows of all j != k: the columns are implicit
    "complete_int": lambda: wl.quio_complete(5, n=200, lo=-40, hi=40),
    # a few zero couplings: mostly single-variable levels, rows read with columns
    "dense_int_zeros": lambda: wl.quio_dense_small(6, n=150, lo=-8, hi=7),
    # path graph plus long-range couplings: single-variable levels, short rows
    "chain_int": lambda: wl.quio_chain(7, n=400, lo=-30, hi=30, n_long=40),
    # fp32 complete graph (fields in fp32, energies refreshed in FP64)
    "complete_float": lambda: wl.batch_instance({"index": 0, "n": 180, "width": 40, "dense": True, "deg": 0,
                                                 "seed": 11}),
}


@pytest.mark.parametrize("case", sorted(SPEC_CASES))
@pytest.mark.parametrize("rule", ALL_RULES)
def test_speculative_windows_equal_level_order(case, rule):
    """Runs of single-variable levels decided 32 at a time by one warp give the
    states, energies, change counts, per-attempt traces and per-sweep energies
    of the level-by-level order, bit for bit, for several launch shapes (float
    energies: bit for bit at the same thread count)."""
    model = Model(SPEC_CASES[case]())
    tmax, tmin = model.default_temperatures()
    S, R, n = 40, 24, model.n
    edt = torch.float64 if model.is_float else torch.int64

    def run(**kw):
        tr = torch.zeros((S, R, n), dtype=torch.int32, device="cuda")
        et = torch.zeros((S, R), dtype=edt, device="cuda")
        out = model.run(rule, S, R, seed=2, t_max=tmax, t_min=tmin, trace=tr, trace_replicas=R,
                        energy_trace=et.data_ptr(), **kw)
        out["trace"], out["energy_trace"] = tr, et
        return out

    ref = run(flags=_lib.SA_FLAG_NO_SPECULATION)
    for extra in [dict(), dict(replicas_per_block=2, threads_per_replica=64),
                  dict(replicas_per_block=1, threads_per_replica=256), dict(flags=_lib.SA_FLAG_STATE_IN_GLOBAL)]:
        got = run(**extra)
        for key in ("states", "accepts", "trace"):
            assert torch.equal(ref[key], got[key]), (case, rule, extra, key)
        for key in ("energies", "energy_trace"):
            if not model.is_float or "threads_per_replica" not in extra:
                assert torch.equal(ref[key], got[key]), (case, rule, extra, key)
            else:
                # FP64 energy partial sums are split over the replica's threads:
                # another thread count rounds them in another order
                torch.testing.assert_close(ref[key], got[key], rtol=1e-12, atol=1e-9)
    # the level-by-level order itself follows the oracle (integer models)
    if not model.is_float and case != "dense_int_zeros":
        om = orc.Model(SPEC_CASES[case]())
        tr = ref["trace"].cpu().numpy()
        res = _oracle_follow(om, rule, S, 2, tmax, tmin, range(4), tr, R)
        for r, x in zip(range(4), res):
            assert x["follow"]["mismatch"] == 0, (case, rule, r, x["follow"])
            assert np.array_equal(x["states"][0], ref["states"][r].cpu().numpy())


def test_state_placement_and_launch_shape_invariance():
    """Global-memory state and other launch shapes give bit-identical results."""
    inst = wl.huio_zipf(4, n=300, n_quad=600, n_cubic=900, n_quartic=200, lo=-9, hi=9)
    model = Model(inst)
    base = model.run("metropolis", 50, 20, seed=9, t_max=300.0, t_min=1.0)
    for kw in [dict(flags=1), dict(replicas_per_block=1, threads_per_replica=64),
               dict(replicas_per_block=3, threads_per_replica=32), dict(flags=1, threads_per_replica=96)]:
        other = model.run("metropolis", 50, 20, seed=9, t_max=300.0, t_min=1.0, **kw)
        assert torch.equal(base["states"], other["states"]), kw
        assert torch.equal(base["energies"], other["energies"]), kw
        assert torch.equal(base["accepts"], other["accepts"]), kw


# ------------------------------------------------------------------ float models
def _float_check(inst, rule, S, R, seed, R_oracle, refresh=0):
    model = Model(inst)
    om = orc.Model(inst)
    tmax, tmin = om.auto_temperatures()
    rep = sa_run_report()
    out = model.run(rule, S, R, seed=seed, t_max=tmax, t_min=tmin, refresh_interval=refresh, report=True)
    st = out["states"]
    e_dev = out["energies"].cpu().numpy()
    e_re = model.energy(st).cpu().numpy()
    np.testing.assert_allclose(e_dev, e_re, rtol=1e-5, atol=1e-6)
    sts = st.cpu().numpy()
    e_orc_of_dev = np.array([om.energy(sts[r]) for r in range(min(R, 64))])
    np.testing.assert_allclose(e_dev[:len(e_orc_of_dev)], e_orc_of_dev, rtol=1e-5, atol=1e-6)
    with cf.ThreadPoolExecutor(max_workers=WORKERS) as ex:
        res = list(ex.map(lambda r: om.run(rule, S, seed, tmax, tmin, r_begin=r, r_end=r + 1), range(R_oracle)))
    e_orc = np.array([x["energy"][0] for x in res])
    p = stats.ks_2samp(e_dev, e_orc).pvalue
    print(f"[parity-float] {rule}: KS p={p:.3g} dev mean={e_dev.mean():.6g} oracle mean={e_orc.mean():.6g} "
          f"drift={out['report']['max_refresh_drift']:.3g}")
    assert p > 0.01
    return out


@pytest.mark.parametrize("rule", ALL_RULES)
def test_quio_float_statistical(rule):
    inst = wl.quio_sparse_wide(11, n=1500, n_edges=12000, lo=0, hi=63)
    _float_check(inst, rule, 100, 512, 3, 96, refresh=25)


@pytest.mark.parametrize("rule", ALL_RULES)
def test_quio_float_wide_range_statistical(rule):
    """Float QUIO over [0,255], the benchmarked range (reduced N = 1500, 12,000
    edges): heat bath through the closed-form window and the register block
    sums (vertex inside, below and above the range), OTM through the quadratic
    vertex, with FP64 refreshes every 10 sweeps; 512 device replicas against 96
    oracle replicas."""
    inst = wl.quio_sparse_wide(11, n=1500, n_edges=12000, lo=0, hi=255)
    S = 100 if rule == "metropolis" else 40
    _float_check(inst, rule, S, 512, 3, 96, refresh=10)


@pytest.mark.parametrize("rule", ALL_RULES)
def test_huio_float_statistical(rule):
    inst = wl.random_interaction(60, 4, 5, n_terms=400, seed=8, integer=False)
    _float_check(inst, rule, 80, 512, 4, 128, refresh=20)


def test_quio_sparse_wide_full_size():
    """Full size sparse float QUIO: N=10,000, z in [0,255], 80,000 edges, 1024
    replicas, 1000 sweeps, FP64 refresh every 50 sweeps, as benchmarked.
    Every replica's energy is within 1e-5 of the FP64 recomputation; 16 oracle
    replicas at full size are KS-compatible with the device replicas."""
    inst = wl.quio_sparse_wide(1)
    model = Model(inst)
    om = orc.Model(inst)
    tmax, tmin = om.auto_temperatures()
    out = model.run("metropolis", 1000, 1024, seed=0, t_max=tmax, t_min=tmin, refresh_interval=50, report=True)
    e_dev = out["energies"].cpu().numpy()
    e_re = model.energy(out["states"]).cpu().numpy()
    np.testing.assert_allclose(e_dev, e_re, rtol=1e-5)
    sts = out["states"].cpu().numpy()
    for r in (0, 511, 1023):
        assert om.energy(sts[r]) == pytest.approx(e_dev[r], rel=1e-5)
    with cf.ThreadPoolExecutor(max_workers=16) as ex:
        res = list(ex.map(lambda r: om.run("metropolis", 1000, 0, tmax, tmin, r_begin=r, r_end=r + 1), range(16)))
    e_orc = np.array([x["energy"][0] for x in res])
    p = stats.ks_2samp(e_dev, e_orc).pvalue
    print(f"[parity-full] C2 metropolis KS p={p:.3g} dev={e_dev.mean():.6g} oracle={e_orc.mean():.6g} "
          f"report={out['report']}")
    assert p > 0.01


# ------------------------------------------------------------------ energy, edge cases, errors
@pytest.mark.parametrize("make", [lambda: wl.quio_dense_small(3),
                                  lambda: wl.random_interaction(30, 4, 5, n_terms=200, seed=1, integer=True),
                                  lambda: wl.random_interaction(30, 3, 5, n_terms=200, seed=2, integer=False),
                                  lambda: wl.quio_sparse_wide(5, n=400, n_edges=1600)])
def test_energy_matches_oracle(make):
    inst = make()
    model = Model(inst)
    om = orc.Model(inst)
    st = wl.initial_states(3, inst, 50)
    e = model.energy(torch.from_numpy(st).cuda()).cpu().numpy()
    want = om.energies(st)
    if model.is_float:
        np.testing.assert_allclose(e, want, rtol=1e-12, atol=1e-9)
    else:
        assert np.array_equal(e, want)


def test_edge_cases():
    # one variable, fixed variables, constant term, S = 1, R = 1
    inst = wl._pack(3, [2, -1, 0], [2, 3, 0], [[0, 1], [1, 1], [], [2]], [3, 2, 5, 7], "i32")
    model = Model(inst)
    om = orc.Model(inst)
    for rule in ALL_RULES:
        for S in (1, 7):
            dev = _device_run(model, rule, S, 1, 4, 10.0, 0.5, trace_R=1)
            x = om.run(rule, S, 4, 10.0, 0.5, r_begin=0, r_end=1, trace=dev["trace"], trace_replicas=1)
            assert x["follow"]["mismatch"] == 0
            assert np.array_equal(x["states"][0], dev["states"][0])
            assert x["energy"][0] == dev["energies"][0]
            assert dev["states"][0][0] == 2 and dev["states"][0][2] == 0
    single = wl._pack(1, [-5], [9], [[0, 0], [0]], [1, -3], "i32")
    m1 = Model(single)
    out = m1.run("heat_bath", 200, 300, seed=1, t_max=5.0, t_min=0.01)
    assert set(out["states"].cpu().numpy().ravel().tolist()) <= {1, 2}   # argmin of z^2 - 3z


def test_init_states_and_host_outputs():
    inst = wl.huio_zipf(6, n=120, n_quad=200, n_cubic=200, n_quartic=50, lo=-4, hi=4)
    model = Model(inst)
    init = wl.initial_states(1, inst, 8)
    trace = torch.zeros((30, 8, model.n), dtype=torch.int32, device="cuda")
    dev_out = model.run("opt_metropolis", 30, 8, seed=2, t_max=50.0, t_min=0.5,
                        init_states=torch.from_numpy(init).cuda(), trace=trace, trace_replicas=8)
    hs = np.zeros((8, model.n), np.int32)
    he = np.zeros(8, np.int64)
    ha = np.zeros(8, np.uint64)
    p = make_params("opt_metropolis", 30, 8, seed=2, t_max=50.0, t_min=0.5, init_states=init)
    sa_run(model.handle, p, hs, he, ha, None)
    assert np.array_equal(hs, dev_out["states"].cpu().numpy())
    assert np.array_equal(he, dev_out["energies"].cpu().numpy())
    om = orc.Model(inst)
    x = om.run("opt_metropolis", 30, 2, 50.0, 0.5, r_begin=0, r_end=8, init_states=init,
               trace=trace.cpu().numpy(), trace_replicas=8)
    assert x["follow"]["mismatch"] == 0, x["follow"]
    assert np.array_equal(x["states"], hs)
    assert np.array_equal(x["energy"], he)
    assert np.array_equal(x["changes"], ha.astype(np.int64))


def test_energy_trace_matches_final():
    inst = wl.quio_dense_small(1)
    model = Model(inst)
    et = torch.zeros((25, 10), dtype=torch.int64, device="cuda")
    trace = torch.zeros((25, 10, model.n), dtype=torch.int32, device="cuda")
    out = model.run("metropolis", 25, 10, seed=3, t_max=50.0, t_min=0.5, energy_trace=et, trace=trace,
                    trace_replicas=10)
    assert torch.equal(et[-1], out["energies"])
    om = orc.Model(inst)
    x = om.run("metropolis", 25, 3, 50.0, 0.5, r_begin=0, r_end=10, energy_trace=True,
               trace=trace.cpu().numpy(), trace_replicas=10)
    assert x["follow"]["mismatch"] == 0, x["follow"]
    assert np.array_equal(x["energy_trace"], et.cpu().numpy())


def test_errors():
    from paper_2511_17245_gb300 import SAError
    inst = wl._pack(2, [-3, -3], [3, 3], [[0, 0, 0, 0, 0, 1]], [1], "i32")   # z0^5 z1
    model = Model(inst)
    with pytest.raises(SAError) as e:
        model.run("opt_metropolis", 2, 2)
    assert e.value.status == 3
    model.run("metropolis", 2, 2, t_max=1.0, t_min=0.1)
    big = wl._pack(2, [-2 ** 20, 0], [2 ** 20, 1], [[0, 0, 0, 1]], [2 ** 10], "i64")
    with pytest.raises(SAError) as e:
        Model(big)
    assert e.value.status == 2
    with pytest.raises(SAError) as e:
        model.run("metropolis", 0, 2)
    assert e.value.status == 1
    with pytest.raises(SAError) as e:
        model.energy(torch.full((1, 2), 9, dtype=torch.int32, device="cuda"))
    assert e.value.status == 1


# ------------------------------------------------------------------ paper models
@pytest.mark.parametrize("rule", ALL_RULES)
def test_multilinear_order_30(rule):
    """E^ML_{30,1} (Sect. 4): terms of 30 distinct variables (general order)."""
    inst = wl.multilinear(100, 30, 1, integer=True)
    _check_int_parity(inst, rule, 200, 16, 3, 8, label="ML p=30 u=1")


@pytest.mark.parametrize("rule", ALL_RULES)
def test_fully_connected_u100(rule):
    """E^FC_{2,100} (Sect. 4), integer-scaled by u^2: dense pairs, z in [-100,100]
    (heat bath over 201 values)."""
    inst = wl.fully_connected(100, 2, 100, integer=True)
    S = 200 if rule != "heat_bath" else 60
    _check_int_parity(inst, rule, S, 8, 5, 4, label="FC p=2 u=100")


def test_energy_trace_equals_oracle():
    """Per-sweep energies (for energy-vs-sweep curves) equal the oracle's."""
    inst = wl.random_interaction(40, 4, 6, n_terms=300, seed=3, integer=True, int_scale=20)
    model = Model(inst)
    om = orc.Model(inst)
    S, R = 50, 6
    et = torch.zeros((S, R), dtype=torch.int64, device="cuda")
    trace = torch.zeros((S, R, model.n), dtype=torch.int32, device="cuda")
    model.run("heat_bath", S, R, seed=2, t_max=500.0, t_min=1.0, energy_trace=et, trace=trace, trace_replicas=R)
    x = om.run("heat_bath", S, 2, 500.0, 1.0, r_begin=0, r_end=R, energy_trace=True, trace=trace.cpu().numpy(),
               trace_replicas=R)
    assert x["follow"]["mismatch"] == 0
    assert np.array_equal(x["energy_trace"], et.cpu().numpy())


# ------------------------------------------------------------------ time-sliced launches
@pytest.mark.parametrize("rule", ALL_RULES)
def test_time_sliced_equals_plain_waves(rule):
    """More replicas than thread groups fit at once (int64 fields of 10,000
    variables: two replicas per SM): the time-sliced cooperative launch, in
    which replicas cut between two groups hand their state over, gives the
    plain waves' results bit for bit, and its traced replicas (replica 1 is
    split between groups 0 and 1) replay exactly against the oracle."""
    inst = wl.quio_sparse_int(13, n=10000, n_edges=60000, lo=-30, hi=200, jmax=4, hmax=40, dmax=3)
    model = Model(inst)
    om = orc.Model(inst)
    tmax, tmin = om.auto_temperatures()
    S, R, TR = 30, 400, 4
    trace = torch.zeros((S, TR, model.n), dtype=torch.int32, device="cuda")
    sliced = model.run(rule, S, R, seed=4, t_max=tmax, t_min=tmin, trace=trace, trace_replicas=TR, report=True,
                       best=True)
    plain = model.run(rule, S, R, seed=4, t_max=tmax, t_min=tmin, flags=_lib.SA_FLAG_NO_TIME_SLICING, report=True,
                      best=True)
    torch.cuda.synchronize()
    assert sliced["report"]["time_sliced"] == 1 and plain["report"]["time_sliced"] == 0, sliced["report"]
    for key in ("states", "energies", "accepts", "best_states", "best_energies"):
        assert torch.equal(sliced[key], plain[key]), key
    res = _oracle_follow(om, rule, S, 4, tmax, tmin, list(range(TR)), trace.cpu().numpy(), TR, best=True)
    st = sliced["states"].cpu().numpy()
    en = sliced["energies"].cpu().numpy()
    bst = sliced["best_states"].cpu().numpy()
    ben = sliced["best_energies"].cpu().numpy()
    for r, x in enumerate(res):
        assert x["follow"]["mismatch"] == 0, (rule, r, x["follow"])
        assert np.array_equal(x["states"][0], st[r]) and x["energy"][0] == en[r]
        # the best state at sweep ends survives the handoffs between groups
        assert np.array_equal(x["best_states"][0], bst[r]) and x["best_energy"][0] == ben[r]


def test_time_sliced_float_benchmark_shape():
    """The 10,000-variable [0,255] fp32 workload with 1024 replicas (the
    benchmark's shape: 608 resident groups) runs time-sliced; every replica's
    energy is within 1e-5 of the FP64 recomputation and the energies match the
    plain waves' by a KS test."""
    inst = wl.quio_sparse_wide(1)
    model = Model(inst)
    tmax, tmin = model.default_temperatures()
    out = {}
    for name, flags in (("sliced", 0), ("plain", _lib.SA_FLAG_NO_TIME_SLICING)):
        out[name] = model.run("heat_bath", 20, 1024, seed=6, t_max=tmax, t_min=tmin, refresh_interval=5,
                              flags=flags, report=True)
    assert out["sliced"]["report"]["time_sliced"] == 1
    e = out["sliced"]["energies"].cpu().numpy()
    np.testing.assert_allclose(e, model.energy(out["sliced"]["states"]).cpu().numpy(), rtol=1e-5)
    assert stats.ks_2samp(e, out["plain"]["energies"].cpu().numpy()).pvalue > 0.01


@pytest.mark.parametrize("rule", ALL_RULES)
def test_speculative_windows_time_sliced(rule):
    """A complete graph (every level one variable) with more replicas than fit
    at once: speculative windows inside a time-sliced launch give the states,
    energies, change counts and best states of the level-by-level plain waves."""
    model = Model(wl.quio_complete(21, n=1500, lo=-40, hi=40))
    tmax, tmin = model.default_temperatures()
    S, R = 20, 2000
    a = model.run(rule, S, R, seed=3, t_max=tmax, t_min=tmin, report=True, best=True)
    b = model.run(rule, S, R, seed=3, t_max=tmax, t_min=tmin, report=True, best=True,
                  flags=_lib.SA_FLAG_NO_SPECULATION | _lib.SA_FLAG_NO_TIME_SLICING)
    assert a["report"]["time_sliced"] == 1 and b["report"]["time_sliced"] == 0, a["report"]
    for key in ("states", "energies", "accepts", "best_states", "best_energies"):
        assert torch.equal(a[key], b[key]), (rule, key)


# ------------------------------------------------------------------ best states at sweep ends
@pytest.mark.parametrize("rule", ALL_RULES)
def test_best_states_integer_replay(rule):
    """Integer models: the best state at sweep ends and its energy equal the
    oracle's (trajectory replay), on a sparse QUIO and a higher-order model;
    host and device outputs agree; the best energy is the best state's energy
    and never above the final one."""
    for inst in (wl.quio_sparse_int(31, n=600, n_edges=3000, lo=-20, hi=20),
                 wl.random_small(32, n=60, max_order=4, lo=-5, hi=5, n_terms=300, coef_type="i32", cmax=6)):
        model = Model(inst)
        om = orc.Model(inst)
        tmax, tmin = om.auto_temperatures()
        S, R, TR = 40, 24, 4
        trace = torch.zeros((S, TR, model.n), dtype=torch.int32, device="cuda")
        out = model.run(rule, S, R, seed=8, t_max=tmax, t_min=tmin, trace=trace, trace_replicas=TR, best=True)
        bst, ben = out["best_states"], out["best_energies"]
        assert torch.equal(model.energy(bst), ben)
        assert bool((ben <= out["energies"]).all())
        # the same run into host buffers
        hs = np.zeros((R, model.n), np.int32)
        he = np.zeros(R, np.int64)
        hb = np.zeros((R, model.n), np.int32)
        hbe = np.zeros(R, np.int64)
        p = make_params(rule, S, R, seed=8, t_max=tmax, t_min=tmin, best_states=hb, best_energies=hbe)
        sa_run(model.handle, p, hs, he)
        assert np.array_equal(hb, bst.cpu().numpy()) and np.array_equal(hbe, ben.cpu().numpy())
        res = _oracle_follow(om, rule, S, 8, tmax, tmin, list(range(TR)), trace.cpu().numpy(), TR, best=True)
        for r, x in enumerate(res):
            assert x["follow"]["mismatch"] == 0, (rule, r, x["follow"])
            assert np.array_equal(x["best_states"][0], hb[r]) and x["best_energy"][0] == hbe[r], (rule, r)


@pytest.mark.parametrize("rule", ALL_RULES)
def test_best_states_float(rule):
    """Float models: the best energy is the FP64 energy of the best state, at
    most the final energy (within the refresh tolerance) and the per-sweep
    energies' minimum (same); speculative windows do not change it."""
    inst = wl.batch_instance({"index": 0, "n": 150, "width": 30, "dense": True, "deg": 0, "seed": 13})
    model = Model(inst)
    tmax, tmin = model.default_temperatures()
    S, R = 60, 32
    et = torch.zeros((S, R), dtype=torch.float64, device="cuda")
    out = model.run(rule, S, R, seed=5, t_max=tmax, t_min=tmin, energy_trace=et, best=True)
    ref = model.run(rule, S, R, seed=5, t_max=tmax, t_min=tmin, best=True, flags=_lib.SA_FLAG_NO_SPECULATION)
    for key in ("best_states", "best_energies"):
        assert torch.equal(out[key], ref[key]), key
    ben = out["best_energies"]
    assert torch.equal(model.energy(out["best_states"]), ben)
    tol = 1e-5 * out["energies"].abs().max().item()
    assert bool((ben <= out["energies"] + tol).all())
    torch.testing.assert_close(ben, et.min(dim=0).values, rtol=1e-5, atol=tol)


def test_best_states_rejected_where_unsupported():
    """Best-state outputs go in pairs, and batches, served requests and the
    allocation-free entry point reject them."""
    from paper_2511_17245_gb300 import (SAError, sa_batch_create, sa_run_noalloc, sa_server_create,
                                        sa_server_destroy, sa_server_submit)
    model = Model(wl.quio_dense_small(0))
    bs = torch.zeros((4, model.n), dtype=torch.int32, device="cuda")
    be = torch.zeros(4, dtype=torch.int64, device="cuda")
    st = torch.zeros((4, model.n), dtype=torch.int32, device="cuda")
    with pytest.raises(SAError) as e:
        sa_run(model.handle, make_params("metropolis", 5, 4, best_states=bs), st, be)
    assert e.value.status == 1
    p = make_params("metropolis", 5, 4, best_states=bs, best_energies=be)
    with pytest.raises(SAError) as e:
        sa_run_noalloc(model.handle, p, st, torch.zeros(4, dtype=torch.int64, device="cuda"))
    assert e.value.status == 3
    with pytest.raises(SAError) as e:
        sa_batch_create([model.handle], [p])
    assert e.value.status == 3
    srv = sa_server_create(1 << 30, 4)
    try:
        with pytest.raises(SAError) as e:
            sa_server_submit(srv, model.handle, p)
        assert e.value.status == 3
    finally:
        sa_server_destroy(srv)
