"""The runtime's host logic, on the CPU: `tests/host_check.cu` compiles the
runtime translation unit into a host program (no GPU involved) that
 - builds plans for seeded synthetic batches -- edge sizes, a 64-setting sweep
   with long and tiled pairs, per-pair settings lists, the swapped direction,
   a strategy table with every form -- and checks that every buffer region of
   every pair and alignment is in place and disjoint, every (pair, gap) is
   aligned once, the settings lists and their by-gap index are right, the
   tiled alignments' tiles come in anti-diagonal order, and the device
   region's byte layout is aligned and disjoint;
 - checks that every pair shape under every strategy-table entry gets an
   alignment form the kernels can run;
 - checks that malformed batches and settings lists are refused with their
   ABI codes and that the int32 overflow bound holds exactly at its edge;
 - saves and loads the strategy table's file through a context built on the
   host (round trips; malformed documents refused, the table unchanged);
 - runs the serving budget's first-fit pool through seeded alloc / release
   sequences against a plain model of the region."""
import os
import shutil
import subprocess

import pytest

from paper_1509_08639_gb300 import _build

HERE = os.path.dirname(os.path.abspath(__file__))


def test_host_logic(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    _build.build()   # the other translation units' objects
    objs = [os.path.join(_build.OUT_DIR, s.replace(".cu", ".o")) for s in _build.SOURCES if s != "runtime.cu"]
    exe = str(tmp_path / "host_check")
    cmd = ([nvcc] + _build.ARCH + ["-O2", "-std=c++17", "-I" + _build.INCLUDE, "-I" + _build.CSRC, "-o", exe,
                                   os.path.join(HERE, "host_check.cu")] + objs + ["-lpthread"])
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([exe, str(tmp_path)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
