"""Bounds audit of the kernels' index arithmetic (CPU).

tests/c/tile_bounds.cc includes the header the kernels take every index
from (paper_2502_00920_gb300/csrc/lbs_tiles.h) and walks the kernels' loops
on the host for every tile shape the library compiles, including four nodes
per thread and the one-node-per-thread frame pieces, over ragged and
degenerate lattices with every combination of periodic and walled axes and
both wall readings: every shared-memory, register, global and side-array
access in bounds and written before it is read, every node written once per
iteration, the TMA boxes on 16-byte boundaries (see the program's header).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_tile_index_arithmetic_stays_in_bounds(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no g++")
    exe = str(tmp_path / "tile_bounds")
    r = subprocess.run([cxx, "-std=c++17", "-O2", "-Wall", "-Wextra", "-Werror",
                        "-I", os.path.join(ROOT, "paper_2502_00920_gb300", "csrc"),
                        os.path.join(ROOT, "tests", "c", "tile_bounds.cc"), "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert run.returncode == 0 and run.stdout.startswith("ok "), run.stdout + run.stderr[-3000:]
