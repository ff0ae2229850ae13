"""The block lookups an ordering indexes once for the factorisation (the
diagonal block of every cluster, every front's row blocks in each of its
columns, the merged position of every block) against the searches they
replace, on grid and grid-free orderings (host C++, no GPU)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2010_06807_gb300", "csrc")


def test_plan_lookups_equal_searches(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path / "plan_index_host")
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "plan_index_host.cpp"), os.path.join(CSRC, "order.cpp"),
                        "-o", exe, "-lpthread"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
