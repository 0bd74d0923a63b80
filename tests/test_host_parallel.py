"""The layout build's host-side parallel passes (csrc/nsn_hostpar.h: the
worker pool, the exclusive scan, the stable counting sort that orders
islands, bodies and constraints, and the union-find that finds the islands)
equal their sequential definitions: a C++ driver compiled with the host
compiler checks them against std::stable_sort, a running sum and a
sequential union-find, with the pool called from two threads at once and
from inside a pass."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parallel_passes_equal_the_sequential_ones(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "host_parallel_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-pthread", "-I", os.path.join(ROOT, "paper_1907_04587_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host_parallel_check.cpp"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
