"""Benchmark: variable-update attempts/s of direct SA on one GB300.

Workload (sparse float QUIO, wide range): N = 10,000 integer variables in
[0, 255]; random graph with 80,000 edges (mean degree 16), J_ij, h_i ~ N(0,1)
fp32, J_ii ~ U[0,1]; 1024 replicas; 1000 sweeps; geometric schedule between
the model-derived temperatures of Sect. 3.4; FP32 fields with an FP64 refresh
every 50 sweeps.  One step = one full run of each of the three rules
(Metropolis, heat bath, optimal-transition Metropolis).  attempts = N R S per
run.  Synthetic, seeded input (there is no dataset in the paper).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun each rank runs the same
workload on its own GPU (replicas only: no collective on the data path) and
`value` is the sum of the ranks' attempts over the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_VARS, N_EDGES, LO, HI = 10_000, 80_000, 0, 255
REPLICAS, SWEEPS, REFRESH = 1024, 1000, 50
RULES = ["metropolis", "heat_bath", "opt_metropolis"]
WORKLOAD = "quio_sparse_wide"
METRIC = "variable-update attempts/s"
UNIT = "attempts/s"
L2_FLUSH_BYTES = 512 << 20
MEAN_DEGREE = 2 * N_EDGES / N_VARS


def _peaks():
    """Measured HBM copy bandwidth and bf16 rate of this machine's GPUs."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def kernel_source_hash():
    """Hash of the CUDA sources and public headers: identifies the build whose
    counters a profile summary records."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2511_17245_gb300", "csrc")
    inc = os.path.join(ROOT, "include")
    files = [os.path.join(csrc, f) for f in sorted(os.listdir(csrc))]
    files += [os.path.join(inc, f) for f in sorted(os.listdir(inc)) if f.endswith(".h")]
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def captured_traffic(rule, sweeps, replicas):
    """DRAM bytes (read + write) per launch of the rule's sweep kernel on this
    workload, from the single-pass ncu capture recorded under profiles/, when
    that capture was taken of these sources at this size; else (None, reason)."""
    path = os.path.join(ROOT, "profiles", f"dram_{rule}_quio_sparse_wide.md")
    if not os.path.exists(path):
        return None, "no capture recorded"
    with open(path) as fh:
        m = re.search(r"traffic: dram_bytes_per_launch=(\d+) sweeps=(\d+) replicas=(\d+) source_hash=(\w+)",
                      fh.read())
    if not m:
        return None, "no capture recorded"
    if int(m.group(2)) != sweeps or int(m.group(3)) != replicas:
        return None, "capture taken at another size"
    if m.group(4) != kernel_source_hash():
        return None, "sources changed since the capture"
    return int(m.group(1)), f"ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch ({os.path.basename(path)})"


def rule_roofline(rule, ms, attempts, change_rate, width, peaks_dev):
    """Roofline of one rule's sweep launch on the benchmark workload, from the
    algorithmic work per attempt (one attempt = one variable visit of one
    replica) and the ceilings measured on this GPU by sa_measure_peaks:
      heat bath   u - l + 1 weights, one exp2 each (Eq. prob_heatbath), against
                  the SFU exp2 rate;
      Metropolis, OTM  replica state in shared memory: read z_k (1 B) and f_k
                  (4 B), and per change write z_k (1 B) and read-modify-write the
                  deg neighbour fields (8 B each), against the shared-memory
                  bandwidth; the changed variable's CSR row (deg x (4 B column +
                  4 B value)) from L2, against the L2-resident copy bandwidth.
    `change_rate` is this rule's measured fraction of attempts that changed
    the variable."""
    sec = ms / 1e3
    deg = MEAN_DEGREE
    if rule == "heat_bath":
        work = attempts * width
        ach = work / sec
        return {"bound": "alu", "unit": "exp2/s", "achieved": ach, "peak": peaks_dev["exp2_per_s"],
                "frac": ach / peaks_dev["exp2_per_s"], "work_per_attempt": f"{width} exp2",
                "peak_source": "sa_measure_peaks exp2 (SFU), measured in this run"}
    smem_b = 5 + change_rate * (1 + 8 * deg)
    l2_b = change_rate * 8 * deg
    smem_gbs = attempts * smem_b / sec / 1e9
    l2_gbs = attempts * l2_b / sec / 1e9
    return {"bound": "smem", "unit": "GB/s", "achieved": smem_gbs, "peak": peaks_dev["smem_gbs"],
            "frac": smem_gbs / peaks_dev["smem_gbs"], "bytes_per_attempt": smem_b,
            "l2": {"achieved": l2_gbs, "peak": peaks_dev["l2_gbs"], "frac": l2_gbs / peaks_dev["l2_gbs"],
                   "bytes_per_attempt": l2_b},
            "change_rate": change_rate,
            "peak_source": "sa_measure_peaks shared-memory and L2-resident copy, measured in this run"}


def _config(extra=None):
    c = {"workload": WORKLOAD, "n_vars": N_VARS, "n_edges": N_EDGES, "range": [LO, HI],
         "replicas": REPLICAS, "sweeps": SWEEPS, "refresh_interval": REFRESH, "rules": RULES,
         "coefficients": "fp32", "l2": "flushed between steps (512 MiB write)"}
    if extra:
        c.update(extra)
    return c


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(value, device=None):
    """Max of a per-rank float over the process group (the job's time is the
    slowest rank's); the value itself on a single process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- CPU oracle leg
def oracle_sample(inst, replicas_per_rule=64, sweeps=2, threads=None):
    """Times the oracle as it stands on the host cores: for each rule,
    `replicas_per_rule` replicas of `sweeps` sweeps of the full-size model,
    replicas spread over host threads.  Returns attempts/s over the three
    rules (equal attempts per rule, as in the GPU step)."""
    import concurrent.futures as cf
    from oracle import oracle as orc
    om = orc.Model(inst)
    tmax, tmin = om.auto_temperatures()
    threads = threads or os.cpu_count() or 1
    total_t = 0.0
    attempts = 0
    per_rule = {}
    for rule in RULES:
        t0 = time.perf_counter()
        with cf.ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(lambda r: om.run(rule, sweeps, 0, tmax, tmin, r_begin=r, r_end=r + 1),
                        range(replicas_per_rule)))
        dt = time.perf_counter() - t0
        total_t += dt
        a = N_VARS * replicas_per_rule * sweeps
        attempts += a
        per_rule[rule] = a / dt
    return {"value": attempts / total_t, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{replicas_per_rule} replicas x {sweeps} sweeps of the full-size model per rule "
                      f"(schedule over {sweeps} sweeps), threads over replicas",
            "per_rule": per_rule, "seconds": total_t}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2511_17245_gb300 import workloads as wl
    from oracle import oracle as orc
    orc.build()
    inst = wl.quio_sparse_wide(1, n=N_VARS, n_edges=N_EDGES, lo=LO, hi=HI)
    for _ in range(args.warmup):
        oracle_sample(inst, replicas_per_rule=16, sweeps=1)
    times, vals = [], []
    res = None
    for _ in range(args.steps):
        res = oracle_sample(inst, replicas_per_rule=args.ref_replicas, sweeps=1)
        vals.append(res["value"])
        times.append(res["seconds"])
    value = float(np.median(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64",
            "data": "synthetic", "config": _config({"sample": res["sample"]}),
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": res["cores"],
                             "sample": res["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- growth directions
def run_batched_vs_plain(torch, hbm_gbs, sample_every=128, sweep_grid=(250, 500, 1000)):
    """4,096 uneven QUIO instances (N log-uniform in [50,2000], range width
    log-uniform in [2,1024], half dense / half sparse with degree 8..64, fp32),
    32 replicas, 1000 sweeps, Metropolis, per-instance temperatures of
    Sect. 3.4.
      batched  one persistent graph-captured launch (autotuned shape);
      plain    one sa_run launch per instance, serialised on one stream, timed
               on every `sample_every`-th dense and sparse instance and scaled;
      time to target  target E* = sum over instances of the plain form's mean
               final energy at 1000 sweeps (same seeds); the batched form is
               run at each sweep count of `sweep_grid` and its time to target
               is the time of the first count whose energy sum is <= E*;
      dense half  the 2,048 dense instances as their own batch: HBM fraction
               of their J-row reads (one row of N-1 (column, value) pairs, 8 B
               each, per accepted change, counted from the change counts);
      other rules  heat bath and OTM, batched vs plain on every 8th dense and
               every 8th sparse instance (512), the plain form timed on the
               same 64 instances as above and scaled."""
    import concurrent.futures as cf
    from paper_2511_17245_gb300 import (Model, make_params, sa_batch_autotune, sa_batch_create, sa_batch_destroy,
                                        sa_batch_get_info, sa_batch_result, sa_batch_run, sa_run)
    from paper_2511_17245_gb300 import workloads as wl
    specs = wl.batch_specs(3)
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        insts = list(ex.map(wl.batch_instance, specs))
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        models = list(ex.map(Model, insts))
    del insts
    create_s = time.perf_counter() - t0
    temps = [m.default_temperatures() for m in models]
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def params_for(S, idx, rule="metropolis"):
        return [make_params(rule, S, 32, seed=0, instance_id=i, t_max=temps[i][0], t_min=temps[i][1])
                for i in idx]

    def timed_batch(idx, S, tune, rule="metropolis"):
        b = sa_batch_create([models[i].handle for i in idx], params_for(S, idx, rule))
        try:
            if tune:
                sa_batch_autotune(b, 10, st.cuda_stream)
            info = sa_batch_get_info(b)
            e0.record(st)
            sa_batch_run(b, st.cuda_stream)
            e1.record(st)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            en = np.zeros((len(idx), 32), np.float64)
            acc = np.zeros((len(idx), 32), np.uint64)
            for j in range(len(idx)):
                sa_batch_result(b, j, None, en[j], acc[j])
            return ms, en, acc, info
        finally:
            sa_batch_destroy(b)

    _progress(f"batched: {len(models)} models built in {create_s:.1f} s")
    everyone = list(range(len(models)))
    grid = {}
    for S in sweep_grid:
        ms, en, acc, info = timed_batch(everyone, S, tune=True)
        _progress(f"batched: {S} sweeps {ms:.0f} ms")
        grid[S] = {"ms": ms, "energy_sum": float(en.mean(axis=1).sum()), "attempts": info["attempts"],
                   "launch_shape": {k: info[k] for k in ("threads_per_replica", "replicas_per_block", "blocks")}}
        if S == 1000:
            en1000 = en
    batched_ms = grid[1000]["ms"]
    att = grid[1000]["attempts"]
    # plain form on a stratified sample (instances alternate dense / sparse)
    sample = list(range(0, len(models), sample_every)) + list(range(1, len(models), sample_every))

    def plain_time(rule, batched_en, pos):
        """Total device time of one sa_run per sampled instance, and the
        largest relative difference of its mean final energy from the batched
        form's (`pos` maps an instance to its row in `batched_en`)."""
        tot, diffs = 0.0, []
        for i in sample:
            m, p = models[i], params_for(1000, [i], rule)[0]
            o_s = torch.empty((32, m.n), dtype=torch.int32, device="cuda")
            o_e = torch.empty(32, dtype=torch.float64, device="cuda")
            e0.record(st)
            sa_run(m.handle, p, o_s, o_e, None, st.cuda_stream)
            e1.record(st)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
            pe = o_e.cpu().numpy()
            diffs.append(abs(batched_en[pos[i]].mean() - pe.mean()) / max(1e-12, abs(pe.mean())))
        return tot, max(diffs)

    plain_ms, rel_max = plain_time("metropolis", en1000, {i: i for i in everyone})
    plain_total_ms = plain_ms * len(models) / len(sample)
    _progress(f"batched: plain sample {plain_ms:.0f} ms")
    target = grid[1000]["energy_sum"]   # equal to the plain form's (same seeds; checked on the sample)
    ttt = next(grid[S]["ms"] for S in sweep_grid if grid[S]["energy_sum"] <= target)
    # dense half alone: HBM roofline of its J-row reads
    dense = [i for i in everyone if specs[i]["dense"]]
    dms, _, dacc, _ = timed_batch(dense, 1000, tune=True)
    row_bytes = sum(float(dacc[j].sum()) * (models[i].n - 1) * 8 for j, i in enumerate(dense))
    dense_gbs = row_bytes / (dms / 1e3) / 1e9
    # heat bath and OTM on a stratified eighth of the instances
    sub = list(range(0, len(models), 16)) + list(range(1, len(models), 16))
    other = {}
    for rule in ("heat_bath", "opt_metropolis"):
        bms, ben, _, binfo = timed_batch(sub, 1000, tune=True, rule=rule)
        pms, pdiff = plain_time(rule, ben, {i: j for j, i in enumerate(sub)})
        p_total = pms * len(sub) / len(sample)
        other[rule] = {"instances": len(sub), "batched_ms": bms, "batched_attempts_per_s": binfo["attempts"] / (bms / 1e3),
                       "plain_ms_estimated": p_total, "plain_attempts_per_s": binfo["attempts"] / (p_total / 1e3),
                       "speedup": p_total / bms, "final_energy_mean_rel_diff_max": float(pdiff),
                       "launch_shape": {k: binfo[k] for k in ("threads_per_replica", "replicas_per_block", "blocks")}}
        _progress(f"batched: {rule} on {len(sub)} instances {bms:.0f} ms, plain estimate {p_total:.0f} ms")
    for m in models:
        m.close()
    return {"workload": "4096 uneven QUIO instances, 32 replicas, 1000 sweeps, metropolis",
            "model_create_s": create_s, "batched_ms": batched_ms, "batched_attempts_per_s": att / (batched_ms / 1e3),
            "plain_ms_estimated": plain_total_ms, "plain_attempts_per_s": att / (plain_total_ms / 1e3),
            "plain_sample": f"every {sample_every}th dense and sparse instance ({len(sample)} launches), "
                            f"scaled by {len(models) / len(sample):.0f}",
            "speedup": plain_total_ms / batched_ms,
            "time_to_target_ms": {"batched": ttt, "plain": plain_total_ms,
                                  "target": "sum of per-instance mean final energies of the plain form, 1000 sweeps",
                                  "batched_sweep_grid": {str(S): {"ms": grid[S]["ms"], "energy_sum": grid[S]["energy_sum"]}
                                                         for S in sweep_grid}},
            "final_energy_mean_rel_diff_max": float(rel_max), "launch_shape": grid[1000]["launch_shape"],
            "dense_half": {"instances": len(dense), "ms": dms, "row_bytes": row_bytes, "achieved_gbs": dense_gbs,
                           "hbm_peak_gbs": hbm_gbs, "frac": dense_gbs / hbm_gbs},
            "other_rules": {"instances": "every 8th dense and every 8th sparse instance (512), 1000 sweeps",
                            "plain_sample": f"the same {len(sample)} instances, scaled by {len(sub) / len(sample):.0f}",
                            **other}}


def _progress(msg):
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def serving_window(max_total_attempts=6e10, max_request_attempts=2e9):
    """The stream's requests in arrival order up to `max_total_attempts`
    attempts (N x replicas x sweeps) in all, leaving out the requests of more
    than `max_request_attempts` attempts (single 32-replica runs of several
    minutes).  Returns the kept requests, their attempts, and what the cap left
    out: the count within the window's range and the share of the whole
    stream's attempts above the cap."""
    from paper_2511_17245_gb300 import workloads as wl
    stream = wl.serving_specs(4)
    out, tot, skipped = [], 0.0, 0
    for sp in stream:
        a = sp["n"] * sp["replicas"] * sp["sweeps"]
        if a > max_request_attempts:
            skipped += 1
            continue
        if out and tot + a > max_total_attempts:
            break
        out.append(sp)
        tot += a
    all_att = sum(sp["n"] * sp["replicas"] * sp["sweeps"] for sp in stream)
    big_att = sum(sp["n"] * sp["replicas"] * sp["sweeps"] for sp in stream
                  if sp["n"] * sp["replicas"] * sp["sweeps"] > max_request_attempts)
    return out, tot, {"skipped_in_window": skipped, "stream_share_of_attempts_above_cap": big_att / all_att,
                      "cap_attempts_per_request": max_request_attempts}


def run_serving(torch, load=0.8):
    """Serving on a window of the request stream (N log-uniform in [100, 50,000],
    ranges [2, 4096], 70% QUIO / 30% HUIO, rules uniform, 100-5000 sweeps, int32
    or fp32 coefficients, 32 replicas): the stream's requests in order (see
    serving_window for what is left out and why).  Through the server
    (150 GB budget, one persistent kernel draining a shared unit queue): all
    requests at once (closed loop: capacity), then Poisson arrivals at `load`
    times that capacity (latency percentiles).  The same requests through the
    batched form (one persistent graph launch per rule / model kind /
    coefficient class group, groups one after another) for comparison, with
    the integer requests' results checked equal between the two forms."""
    import concurrent.futures as cf
    from paper_2511_17245_gb300 import (Model, make_params, sa_batch_create, sa_batch_destroy, sa_batch_result,
                                        sa_batch_run, sa_server_create, sa_server_destroy, sa_server_get_stats,
                                        sa_server_result, sa_server_submit, sa_server_wait)
    from paper_2511_17245_gb300 import workloads as wl
    specs, total_att, window_info = serving_window()
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        insts = list(ex.map(wl.serving_instance, specs))
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        models = list(ex.map(Model, insts))
    del insts
    create_s = time.perf_counter() - t0
    params = []
    for sp, m in zip(specs, models):
        tmax, tmin = m.default_temperatures()
        params.append(make_params(sp["rule"], sp["sweeps"], sp["replicas"], seed=sp["seed"], instance_id=sp["index"],
                                  t_max=tmax, t_min=tmin))
    mean_att = total_att / len(specs)
    served = {}

    def one_pass(rate, keep):
        rng = np.random.default_rng(7)
        srv = sa_server_create(150 << 30, max_running=4096)
        try:
            tickets = []
            start = time.perf_counter()
            arrival = 0.0
            for m, p in zip(models, params):
                if rate:
                    arrival += rng.exponential(1.0 / rate)
                    delay = start + arrival - time.perf_counter()
                    if delay > 0:
                        time.sleep(delay)
                tickets.append(sa_server_submit(srv, m.handle, p))
            for i, t in enumerate(tickets):
                sa_server_wait(srv, t, 3_600_000_000)
                if keep and not models[i].is_float:
                    en = np.zeros(params[i].n_replicas, np.int64)
                    sa_server_result(srv, t, None, en, None)
                    served[i] = en
                else:
                    sa_server_result(srv, t)
            return sa_server_get_stats(srv)
        finally:
            sa_server_destroy(srv)

    _progress(f"serving: {len(specs)} models built in {create_s:.1f} s")
    closed = one_pass(None, True)
    _progress(f"serving: closed loop {closed['attempts_per_s']:.3g} attempts/s")
    rate = load * closed["attempts_per_s"] / mean_att
    open_ = one_pass(rate, False)
    _progress(f"serving: Poisson pass done, p99 {open_['p99_latency_ms']:.0f} ms")

    # batched form on the same requests: one batch per rule, model kind,
    # coefficient class and state placement (a batch keeps all its states in
    # shared memory or all in global memory, so requests whose state does not
    # fit on chip form batches of their own)
    groups = {}
    for i, (sp, m) in enumerate(zip(specs, models)):
        big = m.n * (2 + (4 if m.is_float else 8)) * (1 if m.info["is_quadratic"] else 2) > 48 * 1024
        key = (sp["rule"], bool(m.info["is_quadratic"]), m.is_float, big)
        groups.setdefault(key, []).append(i)
    st = torch.cuda.current_stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batched_ms, mismatch, checked = 0.0, 0, 0
    for key, idx in groups.items():
        b = sa_batch_create([models[i].handle for i in idx], [params[i] for i in idx])
        try:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            sa_batch_run(b, st.cuda_stream)
            e1.record(st)
            torch.cuda.synchronize()
            batched_ms += e0.elapsed_time(e1)
            for j, i in enumerate(idx):
                if i in served:
                    en = np.zeros(params[i].n_replicas, np.int64)
                    sa_batch_result(b, j, None, en, None)
                    checked += 1
                    mismatch += int(not np.array_equal(en, served[i]))
        finally:
            sa_batch_destroy(b)
        _progress(f"serving: batched group {key} ({len(idx)} requests) done")
    batched_wall = time.perf_counter() - t0
    for m in models:
        m.close()
    return {"workload": f"{len(specs)} requests of the 20,000-request stream, in order "
                        f"({total_att:.3g} attempts; largest N {max(sp['n'] for sp in specs)})",
            "window": window_info,
            "model_create_s": create_s,
            "closed_loop": {"attempts_per_s": closed["attempts_per_s"], "p50_latency_ms": closed["p50_latency_ms"],
                            "p99_latency_ms": closed["p99_latency_ms"], "kernel_launches": closed["kernel_launches"]},
            "poisson": {"arrival_rate_per_s": rate, "load": load, "attempts_per_s": open_["attempts_per_s"],
                        "p50_latency_ms": open_["p50_latency_ms"], "p99_latency_ms": open_["p99_latency_ms"],
                        "completed": open_["completed"], "failed": open_["failed"],
                        "device_bytes_peak": open_["device_bytes_peak"]},
            "batched_same_requests": {"groups": len(groups), "kernel_ms": batched_ms,
                                      "attempts_per_s": total_att / (batched_ms / 1e3),
                                      "wall_s_incl_create": batched_wall,
                                      "integer_requests_equal": f"{checked - mismatch}/{checked}"},
            "served_vs_batched": closed["attempts_per_s"] / (total_att / (batched_ms / 1e3)),
            "budget_bytes": 150 << 30}


def run_small_configs(torch, steps=2, warmup=1):
    """The two other single-run workloads, each rule timed with CUDA events
    (median of `steps` runs after `warmup`): the dense 32-variable integer QUIO
    (z in [-8,7], 64 replicas x 1000 sweeps, T 100 -> 0.1) and the Zipf HUIO
    (N = 2,000, z in [-50,50], 8k/20k/5k quadratic/cubic/quartic terms, int32,
    256 replicas x 2000 sweeps, temperatures of Sect. 3.4).  Both fit in L2 and
    shared memory; attempts/s and ns per sweep are reported."""
    from paper_2511_17245_gb300 import Model, make_params, sa_run
    from paper_2511_17245_gb300 import workloads as wl
    st = torch.cuda.current_stream()
    out = {}
    for name, inst, R, S, temps in [("quio_dense_small", wl.quio_dense_small(0), 64, 1000, (100.0, 0.1)),
                                    ("huio_zipf", wl.huio_zipf(2), 256, 2000, None)]:
        m = Model(inst)
        tmax, tmin = temps if temps else m.default_temperatures()
        n = m.n
        states = torch.empty((R, n), dtype=torch.int32, device="cuda")
        energies = torch.empty(R, dtype=torch.int64, device="cuda")
        res = {}
        for rule in RULES:
            p = make_params(rule, S, R, seed=0, t_max=tmax, t_min=tmin)
            for _ in range(warmup):
                sa_run(m.handle, p, states, energies, None, st.cuda_stream)
            ms = []
            for _ in range(steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                sa_run(m.handle, p, states, energies, None, st.cuda_stream)
                e1.record(st)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            t = float(np.median(ms))
            res[rule] = {"ms": t, "attempts_per_s": n * R * S / (t / 1e3), "us_per_sweep": 1e3 * t / S,
                         "mean_final_energy": float(energies.double().mean().item())}
        out[name] = {"n": n, "replicas": R, "sweeps": S, "rules": res}
        m.close()
    return out


# ---------------------------------------------------------------- GPU leg
T_START = time.perf_counter()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--ref-replicas", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rules", default=",".join(RULES))
    ap.add_argument("--sweeps", type=int, default=SWEEPS,
                    help="override for profiling a smaller case (bench numbers use the default)")
    ap.add_argument("--replicas", type=int, default=REPLICAS,
                    help="override for profiling a smaller case (bench numbers use the default)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--time-budget", type=float, default=1500.0,
                    help="seconds the whole run may take; the other configurations' parts that would pass it are skipped")
    ap.add_argument("--quick", action="store_true",
                    help="only the benchmark workload: skip the dense 32-variable and Zipf HUIO runs, the "
                         "batched-vs-plain comparison and serving (several minutes together)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2511_17245_gb300 import (Model, make_params, sa_measure_peaks, sa_model_create, sa_model_destroy,
                                        sa_run, sa_run_report)
    from paper_2511_17245_gb300 import build as pkg_build
    from paper_2511_17245_gb300 import workloads as wl
    pkg_build.build()
    rules = args.rules.split(",")
    # ceilings of this GPU (SFU exp2, FMA, L2-resident copy, shared memory)
    peaks_dev = sa_measure_peaks(torch.cuda.current_stream().cuda_stream)

    inst = wl.quio_sparse_wide(1, n=N_VARS, n_edges=N_EDGES, lo=LO, hi=HI)
    model = Model(inst)
    tmax, tmin = model.default_temperatures()
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    R, S, n = args.replicas, args.sweeps, N_VARS
    states = torch.empty((R, n), dtype=torch.int32, device="cuda")
    energies = torch.empty(R, dtype=torch.float64, device="cuda")
    accepts = torch.empty(R, dtype=torch.int64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    params = {rule: make_params(rule, S, R, seed=rank, t_max=tmax, t_min=tmin, refresh_interval=REFRESH)
              for rule in rules}

    def one_step(record=None):
        for rule in rules:
            if record is not None:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            sa_run(model.handle, params[rule], states, energies, accepts, sptr)
            if record is not None:
                e1.record(stream)
                record.append((rule, e0, e1))

    # first warm-up step: each rule once with a report (launch shape, refresh
    # drift) and its change rate; the rest plain
    change_rates, reports = {}, {}
    for rule in rules:
        rep = sa_run_report()
        p = make_params(rule, S, R, seed=rank, t_max=tmax, t_min=tmin, refresh_interval=REFRESH, report=rep)
        sa_run(model.handle, p, states, energies, accepts, sptr)
        torch.cuda.synchronize()
        change_rates[rule] = float(accepts.double().mean().item()) / (n * S)
        e_re = model.energy(states).double()
        rel = ((energies - e_re).abs() / e_re.abs().clamp_min(1e-300)).max().item()
        reports[rule] = {"threads_per_replica": rep.threads_per_replica, "replicas_per_block": rep.replicas_per_block,
                         "blocks": rep.blocks, "shared_bytes": rep.shared_bytes, "time_sliced": rep.time_sliced,
                         "max_refresh_drift": rep.max_refresh_drift,
                         "final_energy_max_rel_err_vs_fp64_recompute": rel}
    for _ in range(max(0, args.warmup - 1)):
        one_step()
    torch.cuda.synchronize()

    # ---- timed region (device time; L2 flushed between steps, outside the events)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    recs = []
    step_events = []
    acc_sum = 0
    for _ in range(args.steps):
        flush.zero_()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        one_step(recs)
        s1.record(stream)
        step_events.append((s0, s1))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in step_events]
    total_ms = float(sum(step_ms))
    total_ms = max_over_ranks(total_ms, device="cuda")
    attempts_per_run = n * R * S
    attempts = attempts_per_run * len(rules) * args.steps * world
    value = attempts / (total_ms / 1000.0)
    per_rule = {}
    for rule in rules:
        ms = [a.elapsed_time(b) for (rr, a, b) in recs if rr == rule]
        per_rule[rule] = {"ms": float(np.mean(ms)), "attempts_per_s": attempts_per_run / (np.mean(ms) / 1000)}
    # ---- rooflines: every rule against its own ceiling, the dominant (longest)
    # launch as the headline; ceilings measured on this GPU in this run
    peaks, peak_kind = _peaks()
    dom = max(per_rule, key=lambda r: per_rule[r]["ms"])
    per_rule_roof = {}
    for rule in rules:
        per_rule_roof[rule] = rule_roofline(rule, per_rule[rule]["ms"], attempts_per_run, change_rates[rule],
                                            HI - LO + 1, peaks_dev)
        per_rule[rule]["change_rate"] = change_rates[rule]
    roof = dict(per_rule_roof[dom])
    roof["kernel"] = f"{'sweep_sliced_kernel' if reports[dom]['time_sliced'] else 'sweep_kernel'}<{dom}>"
    roof["traffic"], roof["traffic_source"] = captured_traffic(dom, S, R)
    roof["limiter"] = ("ncu: latency-bound (few warps per SM: the replica state fills shared memory; "
                       "per-level barriers; dependent decision chains), not the listed ceiling")
    # ---- e2e through the C ABI with host buffers (model upload + host outputs each step)
    e2e = None
    if rank == 0 and not args.no_e2e:
        hs = torch.empty((R, n), dtype=torch.int32).pin_memory()
        he = torch.empty(R, dtype=torch.float64).pin_memory()
        ha = torch.empty(R, dtype=torch.int64).pin_memory()
        h2d = d2h = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(max(1, min(args.steps, 2))):
            h = sa_model_create(inst["n_vars"], inst["lower"], inst["upper"], inst["term_offsets"],
                                inst["term_vars"], inst["coeffs"], inst["coef_type"])
            from paper_2511_17245_gb300 import sa_model_get_info
            h2d += sa_model_get_info(h)["device_bytes"]
            for rule in rules:
                sa_run(h, params[rule], hs, he, ha, sptr)
                d2h += hs.numel() * 4 + he.numel() * 8 + ha.numel() * 8
            sa_model_destroy(h)
        torch.cuda.synchronize()
        reps = max(1, min(args.steps, 2))
        dt = time.perf_counter() - t0
        e2e = {"value": attempts_per_run * len(rules) * reps / dt, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d / reps), "d2h_bytes_per_step": int(d2h / reps)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(inst, replicas_per_rule=args.ref_replicas, sweeps=1)
        cpu.pop("seconds", None)

    # ---- the other configurations (one GPU, rank 0): the dense 32-variable and
    # Zipf HUIO runs, the batched form against the plain one, and serving; each
    # part is written to stderr as soon as it ends, and a part that fails is
    # recorded with its error instead of ending the benchmark
    extended = None
    if rank == 0 and world == 1 and not args.quick:
        extended = {}
        # (name, function, longest wall time seen for the part, s): a part that
        # could not end within the run's time budget is skipped and said so
        parts = [("small_configs", lambda: run_small_configs(torch), 60),
                 ("batched_vs_plain", lambda: run_batched_vs_plain(torch, float(peaks.get("hbm_gbs", 6800.0))), 600),
                 ("serving", lambda: run_serving(torch), 720)]
        for name, fn, longest in parts:
            elapsed = time.perf_counter() - T_START
            if elapsed + longest > args.time_budget:
                extended[name] = {"skipped": f"{elapsed:.0f} s into the run, the part (up to {longest} s) would pass "
                                             f"the {args.time_budget:.0f} s budget (--time-budget)"}
                print(json.dumps({name: extended[name]}), file=sys.stderr, flush=True)
                continue
            t_part = time.perf_counter()
            try:
                extended[name] = fn()
            except Exception as exc:  # recorded in the line, the benchmark goes on
                extended[name] = {"error": f"{type(exc).__name__}: {exc}"}
            extended[name]["wall_s"] = time.perf_counter() - t_part
            print(json.dumps({name: extended[name]}), file=sys.stderr, flush=True)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 refresh)", "data": "synthetic",
                "config": _config({"parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                                   "replicas": R, "sweeps": S}),
                "per_rule": per_rule, "roofline": roof, "roofline_per_rule": per_rule_roof,
                "peaks_measured": {k: peaks_dev[k] for k in ("exp2_per_s", "fma_per_s", "l2_gbs", "smem_gbs",
                                                            "smem_atomic_per_s", "sms")},
                "peaks_driver": {"hbm_gbs": peaks.get("hbm_gbs"), "source": peak_kind},
                "run_reports": reports, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": len(rules) * args.steps, "clocks": clocks}
        if extended is not None:
            line["extended"] = extended
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
