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
