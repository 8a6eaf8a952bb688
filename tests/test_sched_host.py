"""Host-side checks of the serving loop's policy (serve_policy.h): the workspace
arena (first fit, alignment, coalescing, no overlap) and continuous batching
with admission by device memory (context picked by the oldest request, arrival
order within a context, max batch, memory budget with resident keys counted
once).  Plain C++ built with the host compiler; no GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2112_06396_gb300", "csrc")
SRC = os.path.join(ROOT, "tests", "native", "sched_harness.cpp")


def test_sched_policy(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "sched_harness")
    subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-Werror", "-I", CSRC, SRC, "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    names = [line.split()[1] for line in r.stdout.splitlines() if line.startswith("ok ")]
    assert names == ["arena_basic", "arena_random", "batching_policy", "memory_admission", "fifo_within_context",
                     "random_load"]
