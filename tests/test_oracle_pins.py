"""Pins of the CPU oracle against things other than itself (no GPU needed).

Each test names what fixes the expected value: a published known-answer
vector, a closed form stated in the paper, brute force on a tiny instance, an
independent plain-Python evaluation, or a mathematical invariant.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as orc
from paper_2511_17245_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- Philox
def test_philox_known_answers():
    """Published Philox4x32-10 known-answer vectors (Salmon et al., SC'11)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        vals = [int(x, 16) for x in r]
        out = orc.philox4x32_10(vals[0:4], vals[4:6])
        assert [int(x) for x in out] == vals[6:10]


def test_philox_uniformity():
    """Output words over consecutive counters are uniform (chi-square on 16 bins)."""
    words = np.concatenate([orc.philox4x32_10([k, 7, 3, 0], [5, 9]) for k in range(4000)])
    hist = np.bincount(words >> 28, minlength=16)
    p = stats.chisquare(hist).pvalue
    assert p > 1e-4


# ----------------------------------------------------------------- energy
def _raw_energy(inst, z):
    """Direct evaluation of the unmerged term list (plain Python, exact)."""
    offs, tv, co = inst["term_offsets"], inst["term_vars"], inst["coeffs"]
    is_float = inst["coef_type"] in ("f32", "f64")
    e = 0.0 if is_float else 0
    for t in range(len(offs) - 1):
        prod = 1
        for j in range(offs[t], offs[t + 1]):
            prod *= int(z[tv[j]])
        e += (float(co[t]) * prod) if is_float else int(co[t]) * prod
    return e


@pytest.mark.parametrize("seed", range(6))
def test_energy_matches_unmerged_terms(seed):
    """Merged-model energy equals direct evaluation of the raw (duplicated,
    unsorted) term list: pins merging, sorting and evaluation (Sect. 2)."""
    inst = wl.random_small(seed, n=5, max_order=4, lo=-3, hi=4, n_terms=30,
                           coef_type="i32" if seed % 2 == 0 else "f64")
    m = orc.Model(inst)
    rng = np.random.default_rng(seed)
    for _ in range(20):
        z = rng.integers(inst["lower"], inst["upper"] + 1)
        want = _raw_energy(inst, z)
        got = m.energy(z)
        if m.is_float:
            assert got == pytest.approx(want, rel=1e-12, abs=1e-9)
        else:
            assert got == want


def test_merging_duplicates_zero_and_constant():
    """Permutations of one multiset merge (Sect. 2); zero sums drop; the empty
    multiset is a constant."""
    inst = wl._pack(3, [0, 0, 0], [2, 2, 2],
                    [[0, 1], [1, 0], [2, 2, 1], [1, 2, 2], [2], [], [0, 1, 1]],
                    [3, 4, 5, -5, 7, 11, 0], "i32")
    m = orc.Model(inst)
    offs, tv, ci, _ = m.terms()
    got = {tuple(tv[offs[t]:offs[t + 1]].tolist()): int(ci[t]) for t in range(len(ci))}
    assert got == {(0, 1): 7, (2,): 7}
    assert m.energy([0, 0, 0]) == 11
    assert m.energy([1, 2, 0]) == 11 + 7 * 2


def test_plain_list_instances_take_the_declared_coefficient_type():
    """An instance given as Python lists (coefficients converted to the type it
    declares) evaluates like the hand-expanded polynomial
    E = 3 z0 z1 - 2 z1 z2^2 + z0, for every state of [-2, 2]^3."""
    for ct in ("i32", "i64", "f32", "f64"):
        inst = {"n_vars": 3, "lower": [-2] * 3, "upper": [2] * 3, "term_offsets": [0, 2, 5, 6],
                "term_vars": [0, 1, 1, 2, 2, 0], "coeffs": [3, -2, 1], "coef_type": ct}
        m = orc.Model(inst)
        for z0 in range(-2, 3):
            for z1 in range(-2, 3):
                for z2 in range(-2, 3):
                    assert m.energy([z0, z1, z2]) == 3 * z0 * z1 - 2 * z1 * z2 * z2 + z0, (ct, z0, z1, z2)


def test_fully_connected_ground_energy_closed_form():
    """E^FC ground -N(N+1)/2 (Sect. 4): brute force on a tiny instance and the
    value -5050 the paper quotes for N=100, p=2, u=100 at z = u."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "paper_ground_energies.txt"))
            if l.strip() and not l.startswith("#")]
    fc = [r for r in rows if r[0] == "FC"][0]
    p, u, n, ground = int(fc[1]), int(fc[2]), int(fc[3]), float(fc[4])
    m = orc.Model(wl.fully_connected(n, p, u, integer=False))
    assert m.energy(np.full(n, u)) == pytest.approx(ground, rel=1e-12)
    # integer-scaled, brute force over all states of a small instance
    for (nn, pp, uu) in [(4, 2, 2), (3, 3, 1), (3, 4, 1)]:
        mi = orc.Model(wl.fully_connected(nn, pp, uu, integer=True))
        _, e = mi.enumerate()
        assert e.min() == -(uu ** max(2, pp)) * nn * (nn + 1) // 2


def test_multilinear_ground_energy_closed_form():
    """E^ML ground -N (Sect. 4): brute force and the quoted -100 at N=100."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "paper_ground_energies.txt"))
            if l.strip() and not l.startswith("#") and l.startswith("ML")]
    for r in rows:
        p, u, n, ground = int(r[1]), int(r[2]), int(r[3]), int(r[4])
        m = orc.Model(wl.multilinear(n, p, u, integer=False))
        assert m.energy(np.full(n, u)) == pytest.approx(ground, rel=1e-12)
    for (nn, pp, uu) in [(5, 2, 1), (5, 3, 1), (4, 2, 2)]:
        mi = orc.Model(wl.multilinear(nn, pp, uu, integer=True))
        _, e = mi.enumerate()
        assert e.min() == -nn * uu ** pp


def test_qubo_special_case_matches_textbook():
    """l=0, u=1 (Sect. 2): QUBO energy x^T Q x with the upper triangle."""
    rng = np.random.default_rng(5)
    n = 6
    Q = rng.integers(-5, 6, size=(n, n))
    terms, coefs = [], []
    for i in range(n):
        for j in range(i, n):
            terms.append([i, j] if i != j else [i])
            coefs.append(int(Q[i, j]))
    m = orc.Model(wl._pack(n, np.zeros(n), np.ones(n), terms, coefs, "i64"))
    U = np.triu(Q)
    for s in range(1 << n):
        x = np.array([(s >> i) & 1 for i in range(n)])
        assert m.energy(x) == int(x @ U @ x)


@pytest.mark.parametrize("seed", range(4))
def test_delta_equals_energy_difference(seed):
    """Naive dE over incident terms equals E(z') - E(z) of the full energy."""
    inst = wl.random_small(seed + 10, n=6, max_order=4, lo=-4, hi=4, n_terms=40,
                           coef_type="i64" if seed % 2 == 0 else "f64")
    m = orc.Model(inst)
    rng = np.random.default_rng(seed)
    for _ in range(30):
        z = rng.integers(inst["lower"], inst["upper"] + 1).astype(np.int32)
        k = int(rng.integers(0, inst["n_vars"]))
        v = int(rng.integers(inst["lower"][k], inst["upper"][k] + 1))
        z2 = z.copy()
        z2[k] = v
        want = m.energy(z2) - m.energy(z)
        got = m.delta(z, k, v)
        if m.is_float:
            assert got == pytest.approx(want, abs=1e-9)
        else:
            assert got == want


# ----------------------------------------------------------------- schedule / temperatures
def test_schedule_closed_form():
    """T_i = T_max (T_min/T_max)^((i-1)/(N_sweep-1)) (Sect. 3.1); r = s/(N-1) (Sect. 3.3.3)."""
    t, b, r = orc.schedule(11, 100.0, 0.1)
    assert t[0] == pytest.approx(100.0, rel=1e-15)
    assert t[-1] == pytest.approx(0.1, rel=1e-14)
    ratios = t[1:] / t[:-1]
    assert np.allclose(ratios, (0.1 / 100.0) ** 0.1, rtol=1e-13)
    assert np.all(b == (1.0 / t).astype(np.float32))
    assert np.allclose(r, np.arange(11) / 10.0)
    t1, _, r1 = orc.schedule(1, 5.0, 1.0)
    assert t1[0] == 5.0 and r1[0] == 0.0


def test_auto_temperatures_hand_model():
    """Sect. 3.4 on a hand-computed model: z0,z1 in [-2,3] (z^max=3, width 5);
    E = 3 z0 z1 - 2 z0^2 + 5 z1.  dE_max = max(3*3*5 + 2*25, 3*3*5 + 5*5) = 95;
    dE_min = 2.  T_max = 95/ln 2, T_min = 2/ln 1000."""
    inst = wl._pack(2, [-2, -2], [3, 3], [[0, 1], [0, 0], [1]], [3, -2, 5], "i32")
    tmax, tmin = orc.Model(inst).auto_temperatures()
    assert tmax == pytest.approx(95.0 / math.log(2.0), rel=1e-14)
    assert tmin == pytest.approx(2.0 / math.log(1000.0), rel=1e-14)


# ----------------------------------------------------------------- transition rules
def _tiny_models():
    yield wl.random_small(21, n=3, max_order=3, lo=-1, hi=2, n_terms=8, coef_type="i32", cmax=3)
    yield wl.random_small(22, n=3, max_order=4, lo=[0, -2, -1], hi=[1, 1, 2], n_terms=8,
                          coef_type="f64", cmax=2)


@pytest.mark.parametrize("rule,balanced", [("metropolis", True), ("heat_bath", True),
                                           ("opt_metropolis", False)])
def test_detailed_balance_by_enumeration(rule, balanced):
    """pi(z) P(z->z') = pi(z') P(z'->z) for Metropolis and heat bath; OTM breaks
    it (Sect. 3.3.3).  Exact enumeration, N=3."""
    T = 1.7
    worst = 0.0
    for inst in _tiny_models():
        m = orc.Model(inst)
        states, e = m.enumerate()
        w = np.exp(-(e - e.min()) / T)
        pi = {tuple(s): wi for s, wi in zip(states.tolist(), w)}
        for s in states:
            for k in range(m.n):
                row = m.transition_row(s, k, rule, T, ratio=0.6)
                assert row.sum() == pytest.approx(1.0, abs=1e-12)
                assert np.all(row >= -1e-15)
                for i, pv in enumerate(row):
                    s2 = s.copy()
                    s2[k] = m.lower[k] + i
                    back = m.transition_row(s2, k, rule, T, ratio=0.6)[s[k] - m.lower[k]]
                    lhs, rhs = pi[tuple(s)] * pv, pi[tuple(s2)] * back
                    worst = max(worst, abs(lhs - rhs) / max(lhs, rhs, 1e-300))
    if balanced:
        assert worst < 1e-12
    else:
        assert worst > 1e-3


def _attempt_histogram(m, z, k, rule, temp, ratio, n_draws, seed=123):
    beta = np.float32(1.0 / temp)
    counts = np.zeros(int(m.upper[k] - m.lower[k] + 1), np.int64)
    for r in range(n_draws):
        v = m.attempt(z, k, rule, float(beta), float(np.float32(ratio)), seed, s=5, r=r)
        counts[v - m.lower[k]] += 1
    return counts


@pytest.mark.parametrize("rule", ["metropolis", "heat_bath", "opt_metropolis"])
def test_attempt_sampling_matches_exact_row(rule):
    """The fp32/Philox sampling of one attempt reproduces the exact transition
    row of the rule's definition (chi-square, 20,000 draws)."""
    inst = wl.random_small(31, n=3, max_order=3, lo=-2, hi=3, n_terms=10, coef_type="i32", cmax=3)
    m = orc.Model(inst)
    z = np.array([1, -1, 2], np.int32)
    temp = 3.0
    for k in range(3):
        row = m.transition_row(z, k, rule, float(1.0 / np.float32(1.0 / temp)), ratio=0.4)
        counts = _attempt_histogram(m, z, k, rule, temp, 0.4, 20000)
        exp = row * counts.sum()
        mask = exp > 0
        assert counts[~mask].sum() == 0
        p = stats.chisquare(counts[mask], exp[mask]).pvalue
        assert p > 1e-4, (k, counts, exp)


def test_metropolis_binary_is_single_flip():
    """QUBO case (Sect. 2): the only nonzero change is the flip; acceptance
    frequency equals min(1, exp(-dE/T))."""
    inst = wl._pack(2, [0, 0], [1, 1], [[0], [1], [0, 1]], [2, -1, 3], "i32")
    m = orc.Model(inst)
    z = np.array([0, 1], np.int32)
    dE = m.delta(z, 0, 1)
    assert dE == 5
    counts = _attempt_histogram(m, z, 0, "metropolis", 4.0, 0.0, 20000)
    p_acc = math.exp(-5 / 4.0)
    assert abs(counts[1] / 20000 - p_acc) < 4 * math.sqrt(p_acc * (1 - p_acc) / 20000)


@pytest.mark.parametrize("seed", range(5))
def test_opt_argmin_quadratic_vertex(seed):
    """For dE = c1 d + c2 d^2 with c2 > 0 the argmin over nonzero integer changes
    is the integer nearest the vertex -c1/(2 c2) (exact rational arithmetic),
    or a neighbour when that is the current value."""
    rng = np.random.default_rng(seed)
    n = 4
    inst = wl.quio_sparse_int(seed, n=n, n_edges=5, lo=-20, hi=20)
    m = orc.Model(inst)
    offs, tv, ci, _ = m.terms()
    for _ in range(20):
        z = rng.integers(-20, 21, size=n).astype(np.int32)
        k = int(rng.integers(0, n))
        c1 = m.delta(z, k, z[k] + 1)
        c1m = m.delta(z, k, z[k] - 1) if z[k] > -20 else None
        # recover c2 from two differences: dE(+1) + dE(-1) = 2 c2
        if c1m is None:
            continue
        c2 = Fraction(c1 + c1m, 2)
        c1f = Fraction(c1) - c2
        cands = [v for v in range(-20, 21) if v != z[k]]
        best = min(cands, key=lambda v: (c1f * (v - z[k]) + c2 * (v - z[k]) ** 2, v))
        assert m.argmin_change(z, k) == best


def test_heat_bath_closed_form_multilinear():
    """Multilinear variable: the explicit inverse CDF equals the paper's O(1)
    closed form dz = ceil(P^-1_sum(u, T)) (Eq. inverse_prob) for the same u,
    away from CDF boundaries."""
    inst = wl.multilinear(5, 3, 6, integer=True)
    m = orc.Model(inst)
    rng = np.random.default_rng(3)
    checked = 0
    for trial in range(300):
        z = rng.integers(-6, 7, size=5).astype(np.int32)
        k = int(rng.integers(0, 5))
        temp = float(np.exp(rng.uniform(np.log(0.5), np.log(200.0))))
        beta = np.float32(1.0 / temp)
        T = 1.0 / float(beta)
        a = m.delta(z, k, z[k] + 1)          # dE = a * dz for a multilinear variable
        l, u = int(m.lower[k]), int(m.upper[k])
        words = orc.philox4x32_10([k, 9, trial, 0], [77, 0])
        U = float(((int(words[0]) >> 8) + 1) * 2.0 ** -24)
        v = m.attempt(z, k, "heat_bath", float(beta), 0.0, 77, s=9, r=trial)
        if a == 0 or abs(a * (u - l + 1) / T) > 600:
            continue                      # the formula as printed overflows in double
        X = -(T / a) * math.log(1 - U * (1 - math.exp(-a * (u - l + 1) / T))) - (z[k] - l + 1)
        if abs(X - round(X)) < 1e-6:
            continue
        dz = math.ceil(X)
        assert v == z[k] + dz
        checked += 1
    assert checked > 200


# ----------------------------------------------------------------- runs
def _sweep_params(n_sweeps, s, t_max, t_min):
    frac = s / (n_sweeps - 1) if n_sweeps > 1 else 0.0
    T = t_max * (t_min / t_max) ** frac
    beta = np.float32(1.0 / T)
    ratio = np.float32(s) / np.float32(n_sweeps - 1) if n_sweeps > 1 else np.float32(0)
    return beta, ratio


def _python_attempt(inst, rule, z, k, s, beta, ratio, key, replica):
    """One attempt of Sect. 3.3 on variable k of state z (full-energy
    recomputation for every candidate); returns (new value, near-threshold)."""
    lo, hi = inst["lower"], inst["upper"]
    width = int(hi[k] - lo[k])
    if width == 0:
        return z[k], False
    w = [int(x) for x in orc.philox4x32_10([k, s, replica, 0], key)]
    e0 = _raw_energy(inst, z)

    def dE(v):
        z2 = list(z)
        z2[k] = v
        return _raw_energy(inst, z2) - e0

    if rule == "heat_bath":
        vals = list(range(int(lo[k]), int(hi[k]) + 1))
        des = [dE(v) for v in vals]
        mn = min(des)
        ws = [float(np.exp(-(np.float32(d - mn) * beta), dtype=np.float32)) for d in des]
        thr = ((w[0] >> 8) + 1) * 2.0 ** -24 * sum(ws)
        c = 0.0
        for v, wt in zip(vals, ws):
            c += wt
            if c >= thr:
                return v, False
        return vals[-1], False
    if rule == "opt_metropolis" and np.float32((w[2] >> 8) * 2.0 ** -24) < ratio:
        cands = [v for v in range(int(lo[k]), int(hi[k]) + 1) if v != z[k]]
        prop = min(cands, key=lambda v: (dE(v), v))
    else:
        j = (w[0] * width) >> 32
        off = z[k] - int(lo[k])
        prop = int(lo[k]) + (j + 1 if j >= off else j)
    d = dE(prop)
    if d <= 0:
        return prop, False
    p = float(np.exp(-(np.float32(d) * beta), dtype=np.float32))
    U = (w[1] >> 8) * 2.0 ** -24
    return (prop if U < p else z[k]), abs(U - p) <= 1e-6 * p


def _python_init(inst, key, replica):
    lo, hi = inst["lower"], inst["upper"]
    z = []
    for k in range(inst["n_vars"]):
        w = orc.philox4x32_10([k, 0xFFFFFFFF, replica, 0], key)
        z.append(int(lo[k]) + ((int(w[0]) * int(hi[k] - lo[k] + 1)) >> 32))
    return z


def _python_sa(inst, rule, n_sweeps, seed, t_max, t_min, replica):
    """Independent plain-Python SA of Sect. 3 on a tiny instance: full-energy
    recomputation for every candidate, paper's rules, the documented random
    conventions (Philox counters, 24-bit uniforms, multiply-shift picks).
    Returns the final state, the number of near-threshold decisions and the
    value of z_k after every attempt ([S][N])."""
    n = inst["n_vars"]
    trace = np.zeros((n_sweeps, n), np.int32)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    z = _python_init(inst, key, replica)
    near = 0
    for s in range(n_sweeps):
        beta, ratio = _sweep_params(n_sweeps, s, t_max, t_min)
        for k in range(n):
            z[k], nt = _python_attempt(inst, rule, z, k, s, beta, ratio, key, replica)
            near += nt
            trace[s, k] = z[k]
    return np.array(z), near, trace


@pytest.mark.parametrize("rule", ["metropolis", "heat_bath", "opt_metropolis"])
@pytest.mark.parametrize("window", [2, 5, 32])
def test_speculative_windows_reproduce_sequential_order(rule, window):
    """On a complete graph (every variable depends on every earlier one), the
    attempts of up to `window` consecutive variables decided from the same
    state, kept up to and including the first one that changes its variable,
    give the sequential trajectory of Sect. 3.1 attempt by attempt."""
    inst = wl.quio_complete(9, n=9, lo=-3, hi=3)
    n, S, seed = inst["n_vars"], 6, 0x77
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for rep in range(2):
        ref = _python_sa(inst, rule, S, seed, 40.0, 0.5, rep)[2]
        z = _python_init(inst, key, rep)
        got = np.zeros((S, n), np.int32)
        windows = changes = 0
        for s in range(S):
            beta, ratio = _sweep_params(S, s, 40.0, 0.5)
            i = 0
            while i < n:
                snap = list(z)
                dec = [_python_attempt(inst, rule, snap, k, s, beta, ratio, key, rep)[0]
                       for k in range(i, min(i + window, n))]
                p = next((q for q, v in enumerate(dec) if v != snap[i + q]), len(dec))
                done = min(p + 1, len(dec))   # decisions kept: up to the first change
                for q in range(done):
                    z[i + q] = dec[q]
                    got[s, i + q] = dec[q]
                windows += 1
                changes += p < len(dec)
                i += done
        assert np.array_equal(got, ref), (rule, window, rep)
        assert windows > changes > 0
    # a planted mistake (keeping the decision after the first change) is caught
    if window > 2 and rule == "metropolis":
        z = _python_init(inst, key, 0)
        ref = _python_sa(inst, rule, S, seed, 40.0, 0.5, 0)[2]
        bad = np.zeros((S, n), np.int32)
        for s in range(S):
            beta, ratio = _sweep_params(S, s, 40.0, 0.5)
            snap = list(z)
            for k in range(n):
                z[k] = _python_attempt(inst, rule, snap, k, s, beta, ratio, key, 0)[0]
                bad[s, k] = z[k]
        assert not np.array_equal(bad, ref)


@pytest.mark.parametrize("rule", ["metropolis", "heat_bath", "opt_metropolis"])
def test_run_matches_independent_python_sa(rule):
    """Oracle trajectories equal an independent plain-Python SA (Sect. 3.1:
    sequential index order, geometric schedule) on tiny integer instances."""
    inst = wl.random_small(41, n=4, max_order=3, lo=-2, hi=3, n_terms=12, coef_type="i32", cmax=4)
    m = orc.Model(inst)
    for rep in range(3):
        z_py, near, tr = _python_sa(inst, rule, 12, 0x1234_0000_0042, 20.0, 0.5, rep)
        # the oracle replays the Python trajectory, adopting its decision only
        # within the 1e-6 margin of a threshold; any other difference counts
        follow = np.zeros((12, rep + 1, inst["n_vars"]), np.int32)
        follow[:, rep, :] = tr
        res = m.run(rule, 12, seed=0x1234_0000_0042, t_max=20.0, t_min=0.5, r_begin=rep, r_end=rep + 1,
                    trace=follow, trace_replicas=rep + 1)
        assert res["follow"]["mismatch"] == 0, res["follow"]
        assert res["states"][0].tolist() == z_py.tolist()
        # these seeds meet no decision within the margin, so the oracle's own
        # run (no following) reproduces the Python trajectory as well
        assert near == 0 and res["follow"]["followed"] == 0
        own = m.run(rule, 12, seed=0x1234_0000_0042, t_max=20.0, t_min=0.5, r_begin=rep, r_end=rep + 1)
        assert own["states"][0].tolist() == z_py.tolist()


@pytest.mark.parametrize("rule", ["metropolis", "heat_bath", "opt_metropolis"])
def test_best_state_is_first_lowest_sweep_end(rule):
    """The oracle's best state is, among the independent Python SA's states at
    the ends of the sweeps, the first one of lowest energy (full recompute),
    and its energy is that state's energy."""
    inst = wl.random_small(43, n=5, max_order=3, lo=-2, hi=3, n_terms=14, coef_type="i32", cmax=4)
    m = orc.Model(inst)
    S, seed = 10, 0x55
    for rep in range(3):
        _, near, tr = _python_sa(inst, rule, S, seed, 15.0, 0.5, rep)
        assert near == 0
        ends = [_raw_energy(inst, tr[s].tolist()) for s in range(S)]
        s_best = int(np.argmin(ends))                      # first lowest
        res = m.run(rule, S, seed, 15.0, 0.5, r_begin=rep, r_end=rep + 1, best=True)
        assert res["best_states"][0].tolist() == tr[s_best].tolist(), (rule, rep)
        assert res["best_energy"][0] == ends[s_best] == min(ends)
        assert res["best_energy"][0] <= res["energy"][0]


@pytest.mark.parametrize("rule", ["metropolis", "heat_bath", "opt_metropolis"])
def test_tracked_energy_equals_recomputed(rule):
    for inst in [wl.quio_dense_small(0), wl.random_small(5, n=8, max_order=4, lo=-3, hi=3, n_terms=30, coef_type="f64")]:
        m = orc.Model(inst)
        tmax, tmin = m.auto_temperatures()
        res = m.run(rule, 30, seed=3, t_max=tmax, t_min=tmin, r_begin=0, r_end=4)
        if m.is_float:
            np.testing.assert_allclose(res["energy"], res["energy_recomputed"], rtol=1e-9, atol=1e-9)
        else:
            assert np.array_equal(res["energy"], res["energy_recomputed"])
        assert np.all(res["states"] >= inst["lower"]) and np.all(res["states"] <= inst["upper"])


def test_initial_state_uniform():
    """Random initialisation (Sect. 3.1) is uniform over [l_k, u_k]."""
    inst = wl._pack(1, [-3], [4], [[0]], [0], "i32")
    m = orc.Model(inst)
    res = m.run("metropolis", 1, seed=11, t_max=1.0, t_min=1.0, r_begin=0, r_end=8000,
                init_states=None)
    # the only term has J = 0 and is dropped, so one sweep (every proposal
    # accepted, uniform proposal) keeps the marginal uniform
    hist = np.bincount(res["states"][:, 0] + 3, minlength=8)
    assert stats.chisquare(hist).pvalue > 1e-4


@pytest.mark.parametrize("rule", ["metropolis", "heat_bath"])
def test_fixed_temperature_boltzmann_marginals(rule):
    """At fixed T the chain samples the Boltzmann distribution (balance of
    Metropolis and heat bath): final states of many replicas vs exact
    enumeration, chi-square over all states (N=3, range 4)."""
    inst = wl.random_small(51, n=3, max_order=3, lo=-1, hi=2, n_terms=8, coef_type="i32", cmax=2)
    m = orc.Model(inst)
    states, e = m.enumerate()
    T = 2.5
    pi = np.exp(-(e - e.min()) / T)
    pi /= pi.sum()
    R = 6000
    res = m.run(rule, 40, seed=99, t_max=T, t_min=T, r_begin=0, r_end=R)
    idx = {tuple(s): i for i, s in enumerate(states.tolist())}
    counts = np.zeros(len(states), np.int64)
    for s in res["states"].tolist():
        counts[idx[tuple(s)]] += 1
    exp = pi * R
    mask = exp >= 5
    obs = np.append(counts[mask], counts[~mask].sum())
    ex = np.append(exp[mask], exp[~mask].sum())
    assert stats.chisquare(obs, ex).pvalue > 1e-4


def test_follow_detects_planted_mistake():
    """Following the oracle's own trace gives no mismatch; one planted wrong
    value in the trace is reported at the exact (s, k, r)."""
    inst = wl.quio_dense_small(0)
    m = orc.Model(inst)
    res = m.run("metropolis", 20, seed=0, t_max=100.0, t_min=0.1, r_begin=0, r_end=3, record_trace=True)
    tr = res["trace"]
    ok = m.run("metropolis", 20, seed=0, t_max=100.0, t_min=0.1, r_begin=0, r_end=3,
               trace=tr, trace_replicas=3)
    assert ok["follow"]["mismatch"] == 0
    assert np.array_equal(ok["states"], res["states"])
    bad = tr.copy()
    s, r, k = 7, 1, 13
    bad[s, r, k] = inst["lower"][k] if bad[s, r, k] != inst["lower"][k] else inst["upper"][k]
    out = m.run("metropolis", 20, seed=0, t_max=100.0, t_min=0.1, r_begin=0, r_end=3,
                trace=bad, trace_replicas=3)
    f = out["follow"]
    assert f["mismatch"] >= 1
    assert (f["first_bad_s"], f["first_bad_k"], f["first_bad_r"]) == (s, k, r)
