"""Host-side checks of the kernels' launch decisions (launch_policy.h): the
tensor-core conversion's CTAs per (group, chunk) for a call alone and for n
concurrent calls (the 50 / 76 CTAs of a headline ModUp / ModDown alone, 19 at
n = 8, 7 for a 64-entry batched ModUp), the grouping of batch entries that share
a compressed key, and the NTT autotuner's margin rule.  Plain C++ built with the
host compiler; no GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2112_06396_gb300", "csrc")
SRC = os.path.join(ROOT, "tests", "native", "policy_harness.cpp")


def test_launch_policy(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "policy_harness")
    subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-Werror", "-I", CSRC, SRC, "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    names = [line.split()[1] for line in r.stdout.splitlines() if line.startswith("ok ")]
    assert names == ["tc_grid", "group_cap", "grouping", "tuner"]
