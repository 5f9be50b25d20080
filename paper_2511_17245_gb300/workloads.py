"""Seeded synthetic instance generators for direct SA on QUIO/HUIO.

This module is deliberately free of the method's arithmetic: it only draws
term lists (index multisets with coefficients) and variable bounds.  Both the
CUDA path and the CPU oracle consume its output, so it must never compute an
energy, a field, a temperature or a transition.

An instance is a plain dict:

    n_vars        int
    lower, upper  int64[n_vars]              per-variable bounds l_i <= z_i <= u_i
    term_offsets  int64[n_terms + 1]         CSR over terms
    term_vars     int32[term_offsets[-1]]    index multiset of each term; a
                                             repeated index is a power (z_i^2 ...)
    coeffs        int32/int64/float32/float64[n_terms]
    coef_type     "i32" | "i64" | "f32" | "f64"

Terms may repeat a multiset and may carry a zero coefficient; merging and
dropping are the consumer's job (Sect. 2: permutations of a multiset denote
the same coefficient).

Workload shapes (seeds fixed per workload):
  quio_dense_small  N=32, z in [-8,7], dense symmetric int J in [-10,10],
                    h in [-20,20], J_ii in [0,5]
  quio_sparse_wide  N=10,000, z in [0,255], random graph with 80,000 edges
                    (mean degree 16), fp32 J, h ~ N(0,1), J_ii ~ U[0,1]
  huio_zipf         N=2,000, z in [-50,50], 8,000 quadratic + 20,000 cubic +
                    5,000 quartic terms on distinct variables drawn with
                    Zipf(1.1)-skewed popularity, int J in [-5,5]
  fully_connected   E^FC_{p,u} of Sect. 4 (integer-scaled or float)
  multilinear       E^ML_{p,u} of Sect. 4, periodic
  random_interaction E^RI_{p,u} of Sect. 4, indices drawn with repetition
"""
from __future__ import annotations

import numpy as np

_NP_TYPES = {"i32": np.int32, "i64": np.int64, "f32": np.float32, "f64": np.float64}


def _pack(n_vars, lower, upper, terms, coeffs, coef_type):
    """terms: list of index sequences; coeffs: sequence of numbers."""
    offs = np.zeros(len(terms) + 1, dtype=np.int64)
    lens = np.fromiter((len(t) for t in terms), dtype=np.int64, count=len(terms))
    np.cumsum(lens, out=offs[1:])
    flat = np.zeros(int(offs[-1]), dtype=np.int32)
    pos = 0
    for t in terms:
        flat[pos:pos + len(t)] = t
        pos += len(t)
    return {
        "n_vars": int(n_vars),
        "lower": np.asarray(lower, dtype=np.int64).copy(),
        "upper": np.asarray(upper, dtype=np.int64).copy(),
        "term_offsets": offs,
        "term_vars": flat,
        "coeffs": np.asarray(coeffs, dtype=_NP_TYPES[coef_type]).copy(),
        "coef_type": coef_type,
    }


def _pack_arrays(n_vars, lower, upper, offs, flat, coeffs, coef_type):
    return {
        "n_vars": int(n_vars),
        "lower": np.asarray(lower, dtype=np.int64).copy(),
        "upper": np.asarray(upper, dtype=np.int64).copy(),
        "term_offsets": np.asarray(offs, dtype=np.int64).copy(),
        "term_vars": np.asarray(flat, dtype=np.int32).copy(),
        "coeffs": np.asarray(coeffs, dtype=_NP_TYPES[coef_type]).copy(),
        "coef_type": coef_type,
    }


def _quio_arrays(n, lin_idx, lin_c, diag_idx, diag_c, pi, pj, pc):
    """Assemble linear, self-quadratic and pair terms into CSR arrays."""
    n_lin, n_diag, n_pair = len(lin_idx), len(diag_idx), len(pi)
    offs = np.concatenate([
        np.zeros(1, np.int64),
        np.arange(1, n_lin + 1, dtype=np.int64),
        n_lin + 2 * np.arange(1, n_diag + 1, dtype=np.int64),
        n_lin + 2 * n_diag + 2 * np.arange(1, n_pair + 1, dtype=np.int64),
    ])
    flat = np.concatenate([
        np.asarray(lin_idx, np.int32),
        np.repeat(np.asarray(diag_idx, np.int32), 2),
        np.stack([np.asarray(pi, np.int32), np.asarray(pj, np.int32)], axis=1).reshape(-1),
    ])
    coeffs = np.concatenate([np.asarray(lin_c), np.asarray(diag_c), np.asarray(pc)])
    return offs, flat, coeffs


def quio_dense_small(seed: int = 0, n: int = 32, lo: int = -8, hi: int = 7):
    """Dense integer QUIO: h ~ U{-20..20}, J_ii ~ U{0..5}, J_ij ~ U{-10..10} (i<j)."""
    rng = np.random.default_rng(seed)
    h = rng.integers(-20, 21, size=n)
    d = rng.integers(0, 6, size=n)
    iu, ju = np.triu_indices(n, k=1)
    J = rng.integers(-10, 11, size=len(iu))
    offs, flat, coeffs = _quio_arrays(n, np.arange(n), h, np.arange(n), d, iu, ju, J)
    return _pack_arrays(n, np.full(n, lo), np.full(n, hi), offs, flat, coeffs, "i32")


def quio_complete(seed: int = 0, n: int = 200, lo: int = -40, hi: int = 40):
    """Complete-graph integer QUIO (every pair coupled, so every dependency
    level holds one variable): h ~ U{-20..20}, J_ii ~ U{0..5}, J_ij ~
    U{-10..-1, 1..10} (i<j, never zero)."""
    rng = np.random.default_rng(seed)
    h = rng.integers(-20, 21, size=n)
    d = rng.integers(0, 6, size=n)
    iu, ju = np.triu_indices(n, k=1)
    J = rng.integers(1, 11, size=len(iu)) * rng.choice([-1, 1], size=len(iu))
    offs, flat, coeffs = _quio_arrays(n, np.arange(n), h, np.arange(n), d, iu, ju, J)
    return _pack_arrays(n, np.full(n, lo), np.full(n, hi), offs, flat, coeffs, "i32")


def quio_chain(seed: int = 0, n: int = 300, lo: int = -8, hi: int = 7, n_long: int = 0):
    """Integer QUIO on the path 0-1-...-(n-1) (every level one variable, rows
    of at most two entries), plus n_long random longer-range couplings:
    h ~ U{-20..20}, J_ii ~ U{0..5}, J_ij ~ U{-10..-1, 1..10}."""
    rng = np.random.default_rng(seed)
    h = rng.integers(-20, 21, size=n)
    d = rng.integers(0, 6, size=n)
    pairs = {(k, k + 1) for k in range(n - 1)}
    while len(pairs) < n - 1 + n_long:
        a, b = sorted(int(x) for x in rng.choice(n, size=2, replace=False))
        pairs.add((a, b))
    iu = np.array([a for a, _ in sorted(pairs)], np.int64)
    ju = np.array([b for _, b in sorted(pairs)], np.int64)
    J = rng.integers(1, 11, size=len(iu)) * rng.choice([-1, 1], size=len(iu))
    offs, flat, coeffs = _quio_arrays(n, np.arange(n), h, np.arange(n), d, iu, ju, J)
    return _pack_arrays(n, np.full(n, lo), np.full(n, hi), offs, flat, coeffs, "i32")


def random_graph_edges(rng, n: int, n_edges: int):
    """Distinct undirected edges (i<j) drawn uniformly (Erdos-Renyi G(n, m))."""
    max_edges = n * (n - 1) // 2
    if n_edges > max_edges:
        raise ValueError("too many edges")
    seen = set()
    out_i, out_j = [], []
    while len(out_i) < n_edges:
        need = n_edges - len(out_i)
        a = rng.integers(0, n, size=2 * need + 16)
        b = rng.integers(0, n, size=2 * need + 16)
        for x, y in zip(a.tolist(), b.tolist()):
            if x == y:
                continue
            if x > y:
                x, y = y, x
            key = x * n + y
            if key in seen:
                continue
            seen.add(key)
            out_i.append(x)
            out_j.append(y)
            if len(out_i) == n_edges:
                break
    return np.asarray(out_i, np.int64), np.asarray(out_j, np.int64)


def quio_sparse_wide(seed: int = 1, n: int = 10_000, n_edges: int = 80_000,
                     lo: int = 0, hi: int = 255, coef_type: str = "f32"):
    """Sparse float QUIO on a random graph: J_ij, h_i ~ N(0,1), J_ii ~ U[0,1]."""
    rng = np.random.default_rng(seed)
    ei, ej = random_graph_edges(rng, n, n_edges)
    J = rng.standard_normal(n_edges)
    h = rng.standard_normal(n)
    d = rng.random(n)
    offs, flat, coeffs = _quio_arrays(n, np.arange(n), h, np.arange(n), d, ei, ej, J)
    return _pack_arrays(n, np.full(n, lo), np.full(n, hi), offs, flat, coeffs, coef_type)


def quio_sparse_int(seed: int, n: int, n_edges: int, lo: int, hi: int,
                    jmax: int = 10, hmax: int = 20, dmax: int = 5):
    """Sparse integer QUIO on a random graph (test instances)."""
    rng = np.random.default_rng(seed)
    ei, ej = random_graph_edges(rng, n, n_edges)
    J = rng.integers(-jmax, jmax + 1, size=n_edges)
    h = rng.integers(-hmax, hmax + 1, size=n)
    d = rng.integers(0, dmax + 1, size=n)
    offs, flat, coeffs = _quio_arrays(n, np.arange(n), h, np.arange(n), d, ei, ej, J)
    return _pack_arrays(n, np.full(n, lo), np.full(n, hi), offs, flat, coeffs, "i32")


def _zipf_distinct(rng, probs, size, n_terms):
    """n_terms rows of `size` distinct variables drawn with popularity `probs`."""
    n = len(probs)
    cdf = np.cumsum(probs)
    cdf /= cdf[-1]
    out = np.empty((n_terms, size), dtype=np.int64)
    for t in range(n_terms):
        chosen = []
        while len(chosen) < size:
            v = int(np.searchsorted(cdf, rng.random(), side="right"))
            v = min(v, n - 1)
            if v not in chosen:
                chosen.append(v)
        out[t] = chosen
    return out


def huio_zipf(seed: int = 2, n: int = 2000, n_quad: int = 8000, n_cubic: int = 20_000,
              n_quartic: int = 5000, lo: int = -50, hi: int = 50, cmax: int = 5,
              zipf_s: float = 1.1, coef_type: str = "i32"):
    """Multilinear HUIO with Zipf-skewed variable popularity (distinct vars per term)."""
    rng = np.random.default_rng(seed)
    rank = rng.permutation(n)                     # hubs spread over the index range
    probs = 1.0 / np.power(rank + 1.0, zipf_s)
    blocks, coefs = [], []
    for size, cnt in ((2, n_quad), (3, n_cubic), (4, n_quartic)):
        if cnt == 0:
            continue
        blocks.append(_zipf_distinct(rng, probs, size, cnt))
        if coef_type in ("i32", "i64"):
            coefs.append(rng.integers(-cmax, cmax + 1, size=cnt))
        else:
            coefs.append(rng.uniform(-cmax, cmax, size=cnt))
    terms = [row for b in blocks for row in b.tolist()]
    coeffs = np.concatenate(coefs)
    return _pack(n, np.full(n, lo), np.full(n, hi), terms, coeffs, coef_type)


def fully_connected(n: int, p: int, u: int, integer: bool = True):
    """E^FC_{p,u} = -(1/u^2) sum_{i<j} z_i z_j - (1/u^p) sum_i z_i^p, z in [-u,u].

    With integer=True every coefficient is multiplied by u^max(2,p) so that the
    instance has integer coefficients; its ground energy is then
    -u^max(2,p) N(N+1)/2.
    """
    terms, coefs = [], []
    scale = u ** max(2, p)
    for i in range(n):
        for j in range(i + 1, n):
            terms.append([i, j])
            coefs.append(-(scale // (u * u)) if integer else -1.0 / (u * u))
    for i in range(n):
        terms.append([i] * p)
        coefs.append(-(scale // (u ** p)) if integer else -1.0 / (u ** p))
    return _pack(n, np.full(n, -u), np.full(n, u), terms, coefs, "i64" if integer else "f64")


def multilinear(n: int, p: int, u: int, integer: bool = True):
    """E^ML_{p,u} = -(1/u^p) sum_i z_i z_{i+1} ... z_{i+p-1}, periodic, z in [-u,u].

    integer=True scales by u^p (coefficient -1 per term).
    """
    terms, coefs = [], []
    for i in range(n):
        terms.append([(i + q) % n for q in range(p)])
        coefs.append(-1 if integer else -1.0 / (u ** p))
    return _pack(n, np.full(n, -u), np.full(n, u), terms, coefs, "i64" if integer else "f64")


def random_interaction(n: int, p: int, u: int, n_terms: int = 1000, seed: int = 0,
                       integer: bool = False, int_scale: int = 1000):
    """E^RI_{p,u}: n_terms terms, p indices drawn with repetition, J ~ U[-1,1] / u^p.

    integer=True draws J ~ U{-int_scale..int_scale} instead (test instances).
    """
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, n, size=(n_terms, p))
    if integer:
        J = rng.integers(-int_scale, int_scale + 1, size=n_terms)
        return _pack(n, np.full(n, -u), np.full(n, u), idx.tolist(), J, "i64")
    J = rng.uniform(-1.0, 1.0, size=n_terms) / float(u) ** p
    return _pack(n, np.full(n, -u), np.full(n, u), idx.tolist(), J, "f64")


def quartic_wells(seed: int, n: int = 24, u: int = 1000):
    """Integer HUIO with one tilted double well per variable over z in [-u, u]:
    a_k z^4 - 2 a_k w_k^2 z^2 + c_k z^3 + h_k z (a_k in {1,2,3}, w_k in
    [u/5, 9u/10]), coupled along a ring by J z_i z_j, z_i^2 z_j and z_i^2 z_j^2
    terms.  Every variable's energy difference is a quartic polynomial with up
    to two interior minima, so optimal-transition proposals need the full
    degree-4 argmin and heat-bath draws span 2u + 1 values."""
    rng = np.random.default_rng(seed)
    terms, coefs = [], []
    for k in range(n):
        a = int(rng.integers(1, 4))
        w = int(rng.integers(u // 5, 9 * u // 10 + 1))
        terms += [[k] * 4, [k] * 2, [k] * 3, [k]]
        coefs += [a, -2 * a * w * w, int(rng.integers(-u // 2, u // 2 + 1)), int(rng.integers(-10 ** 8, 10 ** 8 + 1))]
        j = (k + 1) % n
        terms += [[k, j], [k, k, j], [k, k, j, j]]
        coefs += [int(rng.integers(-10 ** 5, 10 ** 5 + 1)), int(rng.integers(-100, 101)), int(rng.integers(-1, 2))]
    return _pack(n, np.full(n, -u), np.full(n, u), terms, coefs, "i64")


def random_small(seed: int, n: int, max_order: int, lo, hi, n_terms: int,
                 coef_type: str = "i32", cmax: int = 5, repeat: bool = True,
                 with_linear: bool = True):
    """Tiny random instance for brute-force checks (indices may repeat)."""
    rng = np.random.default_rng(seed)
    terms, coefs = [], []
    if with_linear:
        for i in range(n):
            terms.append([i])
    for _ in range(n_terms):
        order = int(rng.integers(1, max_order + 1))
        if repeat:
            t = rng.integers(0, n, size=order).tolist()
        else:
            order = min(order, n)
            t = rng.choice(n, size=order, replace=False).tolist()
        terms.append(t)
    nt = len(terms)
    if coef_type in ("i32", "i64"):
        coefs = rng.integers(-cmax, cmax + 1, size=nt)
    else:
        coefs = rng.uniform(-cmax, cmax, size=nt)
    lo_a = np.broadcast_to(np.asarray(lo, np.int64), (n,))
    hi_a = np.broadcast_to(np.asarray(hi, np.int64), (n,))
    return _pack(n, lo_a, hi_a, terms, coefs, coef_type)


def random_bounds(seed: int, n: int, min_width: int, max_width: int, center_span: int = 10):
    """Per-variable bounds with widths log-uniform in [min_width, max_width]."""
    rng = np.random.default_rng(seed)
    w = np.exp(rng.uniform(np.log(min_width), np.log(max_width), size=n)).astype(np.int64)
    w = np.clip(w, min_width, max_width)
    lo = rng.integers(-center_span, center_span + 1, size=n) - w // 2
    return lo.astype(np.int64), (lo + w).astype(np.int64)


def initial_states(seed: int, inst, n_states: int):
    """Uniform random states inside the bounds, int32[n_states, n_vars]."""
    rng = np.random.default_rng(seed)
    lo, hi = inst["lower"], inst["upper"]
    return rng.integers(lo, hi + 1, size=(n_states, inst["n_vars"])).astype(np.int32)


# ---------------------------------------------------------------- batches
def batch_specs(seed: int = 3, n_instances: int = 4096, n_min: int = 50, n_max: int = 2000,
                w_min: int = 2, w_max: int = 1024, deg_min: int = 8, deg_max: int = 64):
    """Uneven batch: per instance N log-uniform in [n_min, n_max], range width
    log-uniform in [w_min, w_max] (values 0..width-1), alternating dense / sparse
    (degree U{deg_min..deg_max}).  Returns small spec dicts; batch_instance()
    materialises one."""
    rng = np.random.default_rng(seed)
    specs = []
    for idx in range(n_instances):
        n = int(np.exp(rng.uniform(np.log(n_min), np.log(n_max))))
        w = int(np.exp(rng.uniform(np.log(w_min), np.log(w_max))))
        dense = (idx % 2 == 0)
        deg = int(rng.integers(deg_min, deg_max + 1))
        specs.append({"index": idx, "n": n, "width": max(2, w), "dense": dense, "deg": deg,
                      "seed": int(rng.integers(0, 2 ** 31))})
    return specs


def batch_instance(spec, as_terms: bool = False):
    """One batch instance: fp32 J, h ~ N(0,1), J_ii ~ U[0,1], z in [0, width-1].
    Dense instances come as {"h", "J"} (symmetric n x n matrix) unless
    as_terms=True; sparse ones always as a term list."""
    rng = np.random.default_rng(spec["seed"])
    n, w = spec["n"], spec["width"]
    lower, upper = np.zeros(n, np.int64), np.full(n, w - 1, np.int64)
    h = rng.standard_normal(n).astype(np.float32)
    d = rng.random(n).astype(np.float32)
    if spec["dense"]:
        A = rng.standard_normal((n, n)).astype(np.float32)
        J = np.triu(A, 1)
        J = J + J.T
        J[np.arange(n), np.arange(n)] = d
        if not as_terms:
            return {"n_vars": n, "lower": lower, "upper": upper, "h": h, "J": J, "coef_type": "f32"}
        iu, ju = np.triu_indices(n, k=1)
        offs, flat, coeffs = _quio_arrays(n, np.arange(n), h, np.arange(n), d, iu, ju, J[iu, ju])
        return _pack_arrays(n, lower, upper, offs, flat, coeffs, "f32")
    m = min(n * spec["deg"] // 2, n * (n - 1) // 2)
    iu, ju = random_graph_edges(rng, n, m)
    Jv = rng.standard_normal(len(iu)).astype(np.float32)
    offs, flat, coeffs = _quio_arrays(n, np.arange(n), h, np.arange(n), d, iu, ju, Jv)
    return _pack_arrays(n, lower, upper, offs, flat, coeffs, "f32")


# ---------------------------------------------------------------- serving stream
def _zipf_rows(rng, n, size, count, zipf_s=1.1):
    """count rows of `size` distinct variables with Zipf popularity (vectorised)."""
    rank = rng.permutation(n)
    p = 1.0 / np.power(rank + 1.0, zipf_s)
    p /= p.sum()
    rows = rng.choice(n, size=(count, size), p=p)
    for _ in range(64):
        srt = np.sort(rows, axis=1)
        bad = np.any(srt[:, 1:] == srt[:, :-1], axis=1)
        if not bad.any():
            break
        rows[bad] = rng.choice(n, size=(int(bad.sum()), size), p=p)
    srt = np.sort(rows, axis=1)
    keep = ~np.any(srt[:, 1:] == srt[:, :-1], axis=1)
    return rows[keep]


def serving_specs(seed: int = 4, n_requests: int = 20_000, n_min: int = 100, n_max: int = 50_000,
                  w_min: int = 2, w_max: int = 4096, s_min: int = 100, s_max: int = 5000, replicas: int = 32):
    """Request stream: 70% sparse QUIO (degree U{8..64}; dense when N <= 4096 with
    probability 0.1), 30% HUIO with the Zipf structure of huio_zipf scaled to N;
    N, range width and sweep count log-uniform; rule uniform; coefficients half
    int32 U{-5..5}, half fp32 N(0,1); 32 replicas."""
    rng = np.random.default_rng(seed)
    rules = ["metropolis", "heat_bath", "opt_metropolis"]
    out = []
    for i in range(n_requests):
        n = int(np.exp(rng.uniform(np.log(n_min), np.log(n_max))))
        w = int(np.exp(rng.uniform(np.log(w_min), np.log(w_max))))
        s = int(np.exp(rng.uniform(np.log(s_min), np.log(s_max))))
        huio = rng.random() < 0.3
        dense = (not huio) and n <= 4096 and rng.random() < 0.1
        out.append({"index": i, "n": n, "width": max(2, w), "sweeps": s, "huio": bool(huio), "dense": bool(dense),
                    "deg": int(rng.integers(8, 65)), "rule": rules[int(rng.integers(0, 3))],
                    "int": bool(rng.random() < 0.5), "replicas": replicas, "seed": int(rng.integers(0, 2 ** 31))})
    return out


def serving_instance(spec):
    """Materialises one request's model (term list, or dense h/J for dense QUIO)."""
    rng = np.random.default_rng(spec["seed"])
    n, w = spec["n"], spec["width"]
    lo = -(w // 2)
    lower, upper = np.full(n, lo, np.int64), np.full(n, lo + w - 1, np.int64)
    ct = "i32" if spec["int"] else "f32"

    def coef(k):
        if spec["int"]:
            return rng.integers(-5, 6, size=k)
        return rng.standard_normal(k).astype(np.float32)

    if spec["huio"]:
        nq, nc, n4 = 4 * n, 10 * n, 5 * n // 2
        blocks = [_zipf_rows(rng, n, 2, nq), _zipf_rows(rng, n, 3, nc), _zipf_rows(rng, n, 4, n4)]
        offs = [np.zeros(1, np.int64)]
        flat, cs = [], []
        pos = 0
        for b in blocks:
            k, sz = b.shape
            offs.append(pos + sz * np.arange(1, k + 1, dtype=np.int64))
            pos += k * sz
            flat.append(b.reshape(-1).astype(np.int32))
            cs.append(coef(k))
        return _pack_arrays(n, lower, upper, np.concatenate(offs), np.concatenate(flat), np.concatenate(cs), ct)
    h = coef(n)
    d = rng.integers(0, 6, size=n) if spec["int"] else rng.random(n).astype(np.float32)
    if spec["dense"]:
        iu, ju = np.triu_indices(n, k=1)
        J = np.zeros((n, n), np.int32 if spec["int"] else np.float32)
        J[iu, ju] = coef(len(iu))
        J[np.arange(n), np.arange(n)] = d
        return {"n_vars": n, "lower": lower, "upper": upper, "h": h, "J": J, "coef_type": ct}
    mdeg = min(n * spec["deg"] // 2, n * (n - 1) // 2)
    iu, ju = random_graph_edges(rng, n, mdeg)
    offs, flat, coeffs = _quio_arrays(n, np.arange(n), h, np.arange(n), d, iu, ju, coef(len(iu)))
    return _pack_arrays(n, lower, upper, offs, flat, coeffs, ct)
