"""The seeded workload generators produce the recipes their docstrings state
(sizes, bounds, term structure, value ranges), so the benchmark and the parity
tests run on the inputs they claim."""
import numpy as np

from paper_2511_17245_gb300 import workloads as wl


def _terms(inst):
    offs, tv = inst["term_offsets"], inst["term_vars"]
    return [tv[offs[t]:offs[t + 1]] for t in range(len(offs) - 1)]


def test_quio_sparse_wide_recipe():
    inst = wl.quio_sparse_wide(1)
    n = inst["n_vars"]
    assert n == 10_000 and inst["coef_type"] == "f32" and inst["coeffs"].dtype == np.float32
    assert np.all(inst["lower"] == 0) and np.all(inst["upper"] == 255)
    terms, c = _terms(inst), inst["coeffs"]
    lin = [i for i, t in enumerate(terms) if len(t) == 1]
    diag = [i for i, t in enumerate(terms) if len(t) == 2 and t[0] == t[1]]
    pair = [i for i, t in enumerate(terms) if len(t) == 2 and t[0] != t[1]]
    assert len(lin) == n and len(diag) == n and len(pair) == 80_000 and len(terms) == 2 * n + 80_000
    keys = {(min(terms[i]), max(terms[i])) for i in pair}
    assert len(keys) == 80_000                                    # distinct edges
    assert np.all((c[diag] >= 0) & (c[diag] < 1))                 # J_ii ~ U[0,1)
    for sel in (lin, pair):                                      # N(0,1)
        x = c[sel].astype(np.float64)
        assert abs(x.mean()) < 0.05 and abs(x.std() - 1) < 0.05
    deg = np.bincount(np.concatenate([terms[i] for i in pair]), minlength=n)
    assert deg.mean() == 16 and deg.max() < 64


def test_huio_zipf_recipe():
    inst = wl.huio_zipf(2)
    assert inst["n_vars"] == 2000 and inst["coef_type"] == "i32"
    assert np.all(inst["lower"] == -50) and np.all(inst["upper"] == 50)
    terms = _terms(inst)
    sizes = np.bincount([len(t) for t in terms])
    assert sizes[2] == 8000 and sizes[3] == 20_000 and sizes[4] == 5000 and len(terms) == 33_000
    assert all(len(set(t.tolist())) == len(t) for t in terms)     # distinct variables: multilinear
    c = inst["coeffs"]
    assert np.all(np.abs(c) <= 5)
    inc = np.bincount(np.concatenate(terms), minlength=2000)
    assert inc.max() > 20 * inc.mean()                            # Zipf-skewed popularity


def test_quio_dense_small_recipe():
    inst = wl.quio_dense_small(0)
    assert inst["n_vars"] == 32 and np.all(inst["lower"] == -8) and np.all(inst["upper"] == 7)
    terms, c = _terms(inst), inst["coeffs"]
    pair = [i for i, t in enumerate(terms) if len(t) == 2 and t[0] != t[1]]
    assert len(pair) == 32 * 31 // 2
    assert np.all(np.abs(c[pair]) <= 10)


def test_batch_and_serving_streams():
    specs = wl.batch_specs(3)
    assert len(specs) == 4096
    n = np.array([s["n"] for s in specs])
    w = np.array([s["width"] for s in specs])
    assert n.min() >= 50 and n.max() <= 2000 and w.min() >= 2 and w.max() <= 1024
    assert [s["dense"] for s in specs[:4]] == [True, False, True, False]
    req = wl.serving_specs(4, n_requests=4000)
    huio = np.mean([r["huio"] for r in req])
    assert 0.27 < huio < 0.33
    assert all(r["replicas"] == 32 and 100 <= r["n"] <= 50_000 and 100 <= r["sweeps"] <= 5000 for r in req)
    assert {r["rule"] for r in req} == {"metropolis", "heat_bath", "opt_metropolis"}
