"""Persistent-kernel grid sizing (host logic, no GPU): the resident blocks per
SM are cached per kernel and per device, and every call forms its grid from
its own device's SM count (csrc/ptf_grid.h, used by ptf_launch.cuh)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs a host C++ compiler")
def test_grid_sizing_per_device(tmp_path):
    exe = str(tmp_path / "grid_check")
    src = os.path.join(ROOT, "tests", "grid_sizing_check.cpp")
    inc = os.path.join(ROOT, "paper_2205_03090_gb300", "csrc")
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", inc, src, "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "grid sizing ok" in r.stdout
