"""Host logic of the automatic launch shape: spare thread slots of a block go
to the replicas only when a model has update lists longer than the inline
limit, never push a block past 512 threads, and cap a replica at 256 threads."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CASES = [
    # tpr, max_link_len, heavy_links, replicas, replicas_per_block, sms -> expected tpr
    (32, 13707, 8, 256, 0, 152, 256),    # Zipf hubs, 2 replicas per SM: 256 threads each
    (128, 35, 64, 1024, 0, 152, 128),    # short rows: unchanged
    (32, 64, 64, 32, 0, 152, 32),        # longest row exactly at the inline limit: unchanged
    (32, 65, 64, 32, 0, 152, 256),       # one link past it
    (32, 999, 64, 1024, 0, 152, 64),     # 7 replicas per block: 512 / 7 -> 64
    (32, 999, 64, 1024, 3, 152, 160),    # caller's 3 replicas per block: 512 / 3 -> 160
    (32, 999, 64, 100000, 0, 152, 32),   # 15 replicas per block (cap): 512 / 15 -> 32
    (256, 999, 64, 4, 0, 152, 256),      # already at the cap
]


def test_grow_threads_per_replica(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    src = tmp_path / "shape.cpp"
    lines = ['#include "sa_internal.h"', "#include <cstdio>", "int main() {"]
    for c in CASES:
        lines.append(f'  std::printf("%d\\n", sa::grow_threads_per_replica({c[0]}, {c[1]}, {c[2]}, {c[3]}, {c[4]}, {c[5]}));')
    lines.append("  return 0; }")
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "shape"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_2511_17245_gb300", "csrc"),
                    str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    got = [int(x) for x in out]
    assert got == [c[6] for c in CASES]
    for c, g in zip(CASES, got):
        per_block = c[4] if c[4] > 0 else max(1, min(15, -(-c[3] // c[5])))
        assert g % 32 == 0 and g <= 256 and (g == c[0] or per_block * g <= 512)


def _compile_and_run(tmp_path, body):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    src = tmp_path / "plan.cpp"
    src.write_text('#include "sa_internal.h"\n#include <cstdio>\nint main() {\n' + body + "\n  return 0; }\n")
    exe = tmp_path / "plan"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_2511_17245_gb300", "csrc"),
                    str(src), "-o", str(exe)], check=True)
    return subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()


def test_plan_run_shape_benchmark_workload(tmp_path):
    """The 10,000-variable [0,255] fp32 workload (43 levels) with 1024 replicas on
    152 SMs and 227 KB of shared memory per block: 128 threads per replica,
    51,856 bytes of state each, 4 replicas per block, 256 blocks."""
    body = """
  sa::PlanModel m{10000, 43, sa::KIND_QUIO, 1, 1, 40, 10000};
  sa::RunPlan p{};
  const char* err = sa::plan_run_shape(m, 1024, 0, 0, false, 152, 232448, &p);
  std::printf("%d %d %d %d %lld %lld %d %d %d %d %d %d\\n", err == nullptr, p.tpr, p.rpc, p.blocks,
              (long long)p.rep_bytes, (long long)p.shared_bytes, p.in_global, p.off_cache, p.off_ctl,
              p.off_list, p.off_red, p.off_lvl);
  err = sa::plan_run_shape(m, 1024, 0, 0, true, 152, 232448, &p);
  std::printf("%d %d %d %lld\\n", err == nullptr, p.in_global, p.rpc, (long long)p.shared_bytes);
  err = sa::plan_run_shape(m, 1024, 48, 0, false, 152, 232448, &p);
  std::printf("%d\\n", err == nullptr);
  err = sa::plan_run_shape(m, 1024, 128, 5, false, 152, 232448, &p);
  std::printf("%d\\n", err == nullptr);
"""
    out = _compile_and_run(tmp_path, body)
    assert out[:12] == ["1", "128", "4", "256", "51856", "207424", "0", "10000", "50000", "50112", "51648", "51680"]
    assert out[12:16] == ["1", "1", "4", "0"]          # forced global state: same shape, no shared memory
    assert out[16] == "0"                               # 48 threads: not whole warps
    assert out[17] == "0"                               # 5 replicas of 51,856 bytes exceed shared memory


def test_plan_schedule_closed_form(tmp_path):
    """Geometric schedule of Sect. 3.1 as fp32 inverse temperatures, OTM ratio
    s/(S-1), the single-sweep case, the Sect. 3.4 defaults and rejections."""
    body = """
  float tab[10];
  const char* err = sa::plan_schedule(0, 0, 5, 100.0, 0.01, nullptr, tab);
  for (int i = 0; i < 10; ++i) std::printf("%.9g\\n", tab[i]);
  std::printf("%d\\n", err == nullptr);
  err = sa::plan_schedule(0, 0, 1, 7.0, 0.5, nullptr, tab);
  std::printf("%.9g %.9g %d\\n", tab[0], tab[1], err == nullptr);
  err = sa::plan_schedule(3.0, 2.0, 2, 0.0, 0.0, nullptr, tab);
  std::printf("%.9g %.9g %d\\n", tab[0], tab[1], err == nullptr);
  double temps[2] = {4.0, -1.0};
  std::printf("%d %d\\n", sa::plan_schedule(0, 0, 2, 0, 0, temps, tab) != nullptr,
              sa::plan_schedule(0, 0, 2, 5.0, 0.0, nullptr, tab) != nullptr);
"""
    out = [float(x) for x in _compile_and_run(tmp_path, body)]
    import numpy as np
    T = 100.0 * (0.01 / 100.0) ** (np.arange(5) / 4)
    np.testing.assert_array_equal(np.array(out[:5], np.float32), (1.0 / T).astype(np.float32))
    np.testing.assert_array_equal(np.array(out[5:10], np.float32), np.float32([0, 0.25, 0.5, 0.75, 1.0]))
    assert out[10] == 1
    assert out[11:14] == [np.float32(1 / 7.0), 0.0, 1]
    tmax, tmin = -3.0 / np.log(0.5), -2.0 / np.log(0.001)
    assert out[14] == np.float32(1 / tmax) and out[15] == np.float32(1 / tmin) and out[16] == 1
    assert out[17:19] == [1, 1]


@pytest.mark.parametrize("R,S,P", [(1024, 1000, 608), (1024, 7, 608), (700, 50, 608), (609, 3, 608),
                                   (5000, 200, 152), (61, 13, 60), (10, 1, 3)])
def test_time_sliced_tasks_cover_every_sweep_once(tmp_path, R, S, P):
    """Time-sliced launch: the chunk-major tasks cover every (replica, sweep)
    pair exactly once in chunks of at most S/16 sweeps, and greedy claiming by
    P groups, simulated with sweeps that cost three times more in the first
    third of the schedule, ends within the list-scheduling bound (total work /
    P + one chunk per dependency wait) and no later than plain waves."""
    import heapq
    out = _compile_and_run(tmp_path, f'  std::printf("%d\\n", sa::slice_chunk_sweeps({S}));')
    K = int(out[0])
    C = -(-S // K)
    assert C <= 16 and (C - 1) * K < S <= C * K
    cost = [3.0 if s < S // 3 else 1.0 for s in range(S)]
    seen = set()
    finish = {}
    heap = [(0.0, p) for p in range(P)]
    for q in range(R * C):
        j, r = divmod(q, R)
        s0, s1 = j * K, min(S, (j + 1) * K)
        for s in range(s0, s1):
            assert (r, s) not in seen
            seen.add((r, s))
        t, p = heapq.heappop(heap)
        start = max(t, finish.get((r, j - 1), 0.0))
        finish[(r, j)] = start + sum(cost[s0:s1])
        heapq.heappush(heap, (finish[(r, j)], p))
    assert len(seen) == R * S
    makespan = max(finish.values())
    per_replica = sum(cost)
    max_chunk = max(sum(cost[j * K:(j + 1) * K]) for j in range(C))
    assert makespan <= R * per_replica / P + 2 * max_chunk + 1e-9
    waves = -(-R // P)
    assert makespan <= waves * per_replica + 1e-9
